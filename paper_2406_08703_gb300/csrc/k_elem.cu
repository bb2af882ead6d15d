// Memory-bound stages of the path: MFT matrix generation, OPD, tilt tables,
// phasor build, binning + flat field + Poisson NLL, the gradient reductions
// and Adam.  Each is a coalesced grid-stride kernel over all active slots.
//
// Reductions.  FP64 arithmetic on this GPU runs at a small fraction of the
// FP32 rate, so per-element work stays in FP32 and long sums are carried as
// compensated (hi, lo) FP32 pairs ("double-float": every addition is an exact
// two-sum, about 44 significant bits); FP64 is used only to combine the few
// per-block partials and in the phase-argument reductions, where an FP32
// argument would lose accuracy.  Every reduction has a fixed order (no
// floating-point atomics), so results do not depend on scheduling or on which
// other slots share the launch.
#include <algorithm>
#include <type_traits>

#include "dlx_common.cuh"

namespace dlx {

// ---------------------------------------------------------------------------
// compensated FP32 pairs
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_add(df a, df b) {
    const float s = a.hi + b.hi, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ df df_add(df a, float b) {
    const float s = a.hi + b, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b - bb);
    e += a.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df warp_sum(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    return v;
}

// Block-wide sums of NV compensated pairs in a fixed order; valid in warp 0.
template <int NV>
__device__ void block_sum(df (&v)[NV], df *sh /* [32][NV] */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[wid * NV + i] = v[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = warp_sum(lane < nw ? sh[lane * NV + i] : df{0.f, 0.f});
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// MFT matrices (Sec. 3, two-sided MFT): A[l][k][n] = sqrt(c) exp(-2 pi i t),
// t = (n - (Ni-1)/2)(k - (No-1)/2) c, c = dx du / lambda_l.  The argument is
// formed and reduced to r = t - rint(t) in FP64 before sin/cos, so the phase
// error does not grow with |t|.  AH[l][n][k] = conj(A[l][k][n]).  Built once
// per plan.  FP16 operands hold A times alpha_l = ascale[l] (|A alpha_l| <= 1).
// With sr != 0 (BF16x3 forms) A is split stochastically; AH (adjoint) is split by
// rounding to nearest, or (ah_hi, BF16x3sa form) holds only the stochastically
// rounded hi parts in two planes (re, im).
// Paired forward matrix (hp > 0, FP16 split form; pair_layout in dlx_common.cuh): for n < hn
// the row k of amat holds a = Re A[k][n] at column n and b = Im A[k][n] at column hp + n (times
// alpha_l), split into two planes (hi, lo) of ldk columns.
// Paired adjoint matrix (hpo > 0): for k < hno the row n of amatH holds Re A^H[n][k] = Re A[k][n]
// at column k and Im A^H[n][k] = -Im A[k][n] at column hpo + k, two planes of ldko columns.
template <int F>
__global__ void k_mft_matrices(void *amat, void *amatH, const double *lam, const float *ascale, int nl, int ni,
                               int no, int ldi, int ldo, double dx, double du, uint32_t sr, int ah_hi, int hp,
                               int ldk, int hpo, int ldko) {
    const int P = fmt_planes(F), es = fmt_esize(F);
    const size_t per = (size_t)no * ni, total = per * nl;
    const double cN = 0.5 * (ni - 1), cO = 0.5 * (no - 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int l = (int)(i / per);
        int k = (int)((i % per) / ni), n = (int)(i % ni);
        double c = dx * du / lam[l];
        double t = ((double)n - cN) * ((double)k - cO) * c;
        double r = t - rint(t);
        double s, co;
        sincospi(2.0 * r, &s, &co);
        const double sc = sqrt(c) * (F == FMT_F16X4 ? (double)ascale[l] : 1.0);
        float re = (float)(sc * co), im = (float)(-sc * s);
        char *a = (char *)amat + (size_t)l * P * no * ldi * es;
        if constexpr (F == FMT_F16X4) {
            if (hp > 0) {
                if (2 * n < ni) {  // n < hn: a at column n, b at column hp + n (hi, lo planes)
                    using H = H16<F>;
                    typename H::T *q = (typename H::T *)amat + (size_t)l * 2 * no * ldk + (size_t)k * ldk + n;
                    const size_t pl = (size_t)no * ldk;
                    const typename H::T ah = H::hi(re), bh = H::hi(im);
                    q[0] = ah;
                    q[pl] = H::from(re - H::to(ah));
                    q[hp] = bh;
                    q[pl + hp] = H::from(im - H::to(bh));
                }
            } else {
                store_cplx<F>(a, (size_t)no * ldi, (size_t)k * ldi + n, re, im);
            }
        } else if constexpr (F == FMT_BF16X4) {
            if (sr) {
                store_cplx_sr(a, (size_t)no * ldi, (size_t)k * ldi + n, re, im, ((size_t)l * no + k) * ldi + n,
                              sr ^ 0x2545f491u);
            } else {
                store_cplx<F>(a, (size_t)no * ldi, (size_t)k * ldi + n, re, im);
            }
        } else {
            store_cplx<F>(a, (size_t)no * ldi, (size_t)k * ldi + n, re, im);
        }
        if constexpr (F == FMT_BF16X4) {
            if (ah_hi) {
                unsigned short *ah = (unsigned short *)amatH + (size_t)l * 2 * ni * ldo;
                const uint32_t rb = sr_word(((size_t)l * ni + n) * ldo + k, sr ^ 0x68e31da4u);
                const size_t o = (size_t)n * ldo + k;
                const uint32_t d = cvt_bf16x2_sr(-im, re, rb);  // re with bits 15:0, -im with 31:16
                ah[o] = (unsigned short)d;
                ah[(size_t)ni * ldo + o] = (unsigned short)(d >> 16);
                continue;
            }
        }
        if constexpr (F == FMT_F16X4) {
            if (hpo > 0) {
                if (2 * k < no) {
                    using H = H16<F>;
                    typename H::T *q = (typename H::T *)amatH + (size_t)l * 2 * ni * ldko + (size_t)n * ldko + k;
                    const size_t pl = (size_t)ni * ldko;
                    const typename H::T ah = H::hi(re), bh = H::hi(-im);
                    q[0] = ah;
                    q[pl] = H::from(re - H::to(ah));
                    q[hpo] = bh;
                    q[pl + hpo] = H::from(-im - H::to(bh));
                }
                continue;
            }
        }
        char *ah = (char *)amatH + (size_t)l * P * ni * ldo * es;
        store_cplx<F>(ah, (size_t)ni * ldo, (size_t)n * ldo + k, re, -im);
    }
}

cudaError_t launch_mft_matrices(dlx_plan *p, cudaStream_t st) {
    size_t total = (size_t)p->nl * p->no * p->ni;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)p->sm_count * 16);
    KScope ks(p, KC_MATRICES, 1, st);
    DLX_FMT_DISPATCH(p->fmt, F,
                     k_mft_matrices<F><<<blocks, 256, 0, st>>>(p->amat.ptr, p->amatH.ptr, p->lam_d, p->ascale, p->nl,
                                                               p->ni, p->no, p->ldi, p->ldo, p->dx, p->du, p->sr,
                                                               p->adj1 ? 1 : 0, p->paired ? p->hp : 0, p->ldk,
                                                               p->padj ? p->hpo : 0, p->ldko));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prologue pass, grid (blocks, R), slot r = blockIdx.y:
//  * OPD = OPD_fixed + sum_j c_j Z_j + OPD_pix (Sec. 3: BasisOptic coefficients
//    on a Zernike basis, the fixed mask, and the free per-pixel map);
//  * sum T^2 for the pupil normalisation of BasisOptic(normalise=True): block
//    partials go to npart[r][block] (and max |T| to tpart), and the last block
//    of the slot to finish combines them in a fixed order into
//    pscale[r] = (1 / sqrt(sum T^2), pi_r), pi_r the FP16 operand scale of the
//    phasor (2^-ceil(log2 max |T_hat|)); sum T^2 is carried in compensated FP32
//    pairs, per block and across blocks (fixed order);
//  * clears the slot's FP16 scale maxima (qmax, gmax) of the adjoint;
//  * the separable tilt factors exp(i 2 pi x_n theta / lambda) of every PSF and
//    axis, theta = pos[s] + dither[e], with the argument reduced in FP64;
//  * block 0 writes the normalised spectral weights w_l / sum w.
__global__ void k_prologue(DevParams prm, int nz, int npx, int nl, float *__restrict__ opd, float2 *npart,
                           float *tpart, unsigned int *ncount, float *pscale, float *wnorm,
                           const double *__restrict__ lam, int B, int nse, int ne, int ni, double dx,
                           float2 *__restrict__ tilt, unsigned int *qmax, unsigned int *gmax, double chirp) {
    pdl_wait();
    extern __shared__ float c_sh[];
    __shared__ df sh[32];
    __shared__ bool s_last;
    const int r = blockIdx.y;
    const float *fixed = slot_ptr(prm, POPDF, r), *basis = slot_ptr(prm, PBASIS, r);
    const float *coeff = slot_ptr(prm, PCOEFF, r), *pix = slot_ptr(prm, POPDPIX, r), *T = slot_ptr(prm, PT, r);
    for (int j = threadIdx.x; j < nz; j += blockDim.x) c_sh[j] = coeff[j];
    __syncthreads();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    if (qmax)
        for (int i = tid; i < nse; i += nthr) qmax[(size_t)r * nse + i] = 0u;
    if (gmax)
        for (int i = tid; i < B; i += nthr) gmax[(size_t)r * B + i] = 0u;
    df t2[1] = {{0.f, 0.f}};
    float tmax = 0.f;
    // one thread per pupil pixel: the Zernike terms go into eight partial sums (eight basis
    // loads in flight), added in a fixed order
    for (int i = tid; i < npx; i += nthr) {
        float part[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) part[q] = 0.f;
        int j = 0;
        for (; j + 7 < nz; j += 8) {
            float z[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) z[q] = __ldg(basis + (size_t)(j + q) * npx + i);
#pragma unroll
            for (int q = 0; q < 8; ++q) part[q] = fmaf(c_sh[j + q], z[q], part[q]);
        }
        for (int q = 0; j < nz; ++j, ++q) part[q] = fmaf(c_sh[j], __ldg(basis + (size_t)j * npx + i), part[q]);
        float o = fixed ? __ldg(fixed + i) : 0.f;
        o += ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
        if (pix) o += __ldg(pix + i);
        opd[(size_t)r * npx + i] = o;
        const float t = __ldg(T + i);
        t2[0] = df_add(t2[0], t * t);
        tmax = fmaxf(tmax, fabsf(t));
    }
    // tilt factors of this slot's PSFs: tilt[r B + bl][axis][n]; in the Fresnel regime each also
    // carries its axis' share of the quadratic phase exp(i pi |x|^2 (1/z - 1/f) / lambda), the
    // factor before the transform (separable: x^2 + y^2), chirp = (1/z - 1/f) / 2
    {
        const float *pos = slot_ptr(prm, PPOS, r), *dith = slot_ptr(prm, PDITHER, r);
        const double cN = 0.5 * (ni - 1);
        float2 *tl = tilt + (size_t)r * B * 2 * ni;
        for (int i = tid; i < B * 2 * ni; i += nthr) {
            const int bl = i / (2 * ni), ax = (i / ni) & 1, n = i - (i / ni) * ni;
            const int l = bl / nse, se = bl - l * nse, s = se / ne, e = se - s * ne;
            const double th = (double)pos[2 * s + ax] + (dith ? (double)dith[2 * e + ax] : 0.0);
            const double xn = ((double)n - cN) * dx;
            const double t = (xn * th + chirp * xn * xn) / lam[l];
            float sn, cs;
            sincospif((float)(2.0 * (t - rint(t))), &sn, &cs);
            tl[i] = make_float2(cs, sn);
        }
    }
    __shared__ float s_tmax[32];
    for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    if ((threadIdx.x & 31) == 0) s_tmax[threadIdx.x >> 5] = tmax;
    block_sum<1>(t2, sh);  // its barriers also publish s_tmax
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tmax = fmaxf(tmax, s_tmax[w]);
        npart[(size_t)r * gridDim.x + blockIdx.x] = make_float2(t2[0].hi, t2[0].lo);
        tpart[(size_t)r * gridDim.x + blockIdx.x] = tmax;
        __threadfence();
        s_last = (atomicAdd(ncount + r, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        // every other block's partial is visible (fence before its count); fixed order
        __threadfence();
        df v[1] = {{0.f, 0.f}};
        float m = 0.f;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            const float2 x = __ldcg(npart + (size_t)r * gridDim.x + b);
            v[0] = df_add(v[0], df{x.x, x.y});
            m = fmaxf(m, __ldcg(tpart + (size_t)r * gridDim.x + b));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) s_tmax[threadIdx.x >> 5] = m;
        block_sum<1>(v, sh);  // its barriers also publish s_tmax
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_tmax[w]);
            const float sc = (float)(1.0 / sqrt(df_to_double(v[0])));
            pscale[2 * r] = sc;
            pscale[2 * r + 1] = inv_pow2_ceil(m * sc);
            ncount[r] = 0;  // ready for the next launch
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const float *w = slot_ptr(prm, PW, r);
        df ws{0.f, 0.f};
        for (int l = 0; l < nl; ++l) ws = df_add(ws, w[l]);
        const float wsum = ws.hi + ws.lo;
        for (int l = 0; l < nl; ++l) wnorm[(size_t)r * nl + l] = w[l] / wsum;
    }
}

// Pupil phasor P = T_hat exp(i 2 pi OPD / lambda) ex[nx] ey[ny] (Sec. 3), written
// in the operand form of the contractions.  OPD / lambda is below one cycle for
// the aberrations of interest, so FP32 is exact enough there.  One thread takes
// eight consecutive columns of a row for one wavelength: the common factor
// T_hat exp(i 2 pi OPD / lambda) is formed once and multiplied by the tilt of
// each source and exposure of that wavelength (16- or 32-byte stores per
// plane); columns from Ni up to the padded row length are written as zeros.
// Grid: x over the eight-column groups, y over (slot, wavelength).  Four blocks per SM (64
// registers, a few spilled in the BF16 split form) measured faster than three at 79 registers.
template <int F>
__global__ void __launch_bounds__(256, 4) k_phasor(DevParams prm, const float *__restrict__ opd, const float2 *__restrict__ tilt,
                         const float *__restrict__ invlam, const float *__restrict__ pscale, int B, int nl, int nse,
                         int ne, int ni, int ldi, void *P, uint32_t sr, const float *__restrict__ tmap, float tcoef,
                         uint32_t tmask) {
    pdl_wait();
    const int npx = ni * ni, Pl = fmt_planes(F), es = fmt_esize(F), gpr = ldi >> 3;
    const int r = blockIdx.y / nl, l = blockIdx.y - r * nl;
    const float *T = slot_ptr(prm, PT, r), *op = opd + (size_t)r * npx;
    // FP16 operands hold pi_r P
    const float sc = pscale[2 * r] * (F == FMT_F16X4 ? pscale[2 * r + 1] : 1.f), il = invlam[l];
    const size_t ps = (size_t)ni * ldi;
    // vector loads need 8-wide rows and a 16-byte aligned caller transmission map
    const bool vec = (ni & 7) == 0 && ((uintptr_t)T & 15) == 0;
    for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < ni * gpr; gi += gridDim.x * blockDim.x) {
        const int ny = gi / gpr, nx0 = (gi - ny * gpr) * 8;
        float t[8], o[8];
        if (vec) {
            const float4 *T4 = (const float4 *)(T + (size_t)ny * ni + nx0), *O4 = (const float4 *)(op + (size_t)ny * ni + nx0);
            const float4 ta = __ldg(T4), tb = __ldg(T4 + 1), oa = __ldg(O4), ob = __ldg(O4 + 1);
            t[0] = ta.x; t[1] = ta.y; t[2] = ta.z; t[3] = ta.w; t[4] = tb.x; t[5] = tb.y; t[6] = tb.z; t[7] = tb.w;
            o[0] = oa.x; o[1] = oa.y; o[2] = oa.z; o[3] = oa.w; o[4] = ob.x; o[5] = ob.y; o[6] = ob.z; o[7] = ob.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool in = nx0 + q < ni;
                t[q] = in ? __ldg(T + (size_t)ny * ni + nx0 + q) : 0.f;
                o[q] = in ? __ldg(op + (size_t)ny * ni + nx0 + q) : 0.f;
            }
        }
        // tangent direction of dlx_model_jvp: a = tcoef (2 pi / lambda) t[n] for the masked sources
        float ta[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            ta[q] = (tmap && nx0 + q < ni) ? tcoef * 6.283185307f * il * __ldg(tmap + (size_t)ny * ni + nx0 + q) : 0.f;
        // T_hat exp(i 2 pi OPD / lambda), common to every source and exposure
        float br[8], bi[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            br[q] = 0.f;
            bi[q] = 0.f;
            const float tq = t[q] * sc;
            if (tq != 0.f) {
                float ph = o[q] * il;
                ph -= rintf(ph);
                float sn, cs;
                sincospif(2.f * ph, &sn, &cs);
                br[q] = tq * cs;
                bi[q] = tq * sn;
            }
        }
        for (int se = 0; se < nse; ++se) {
            const int bg = r * B + l * nse + se;
            const float2 *tx = tilt + (size_t)bg * 2 * ni, *ty = tx + ni;
            float2 ex[8];
            if (vec) {
                const float4 *X4 = (const float4 *)(tx + nx0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 x = __ldg(X4 + q);
                    ex[2 * q] = make_float2(x.x, x.y);
                    ex[2 * q + 1] = make_float2(x.z, x.w);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) ex[q] = nx0 + q < ni ? __ldg(tx + nx0 + q) : make_float2(0.f, 0.f);
            }
            const float2 ey = __ldg(ty + ny);
            const bool tan = tmap && ((tmask >> (se / ne)) & 1u);
            float re[8], im[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float cr = br[q], ci = bi[q];
                if (tan) {  // times (1 + i a)
                    const float a = ta[q], nr = cr - a * ci;
                    ci = ci + a * cr;
                    cr = nr;
                }
                const float xr = ex[q].x * ey.x - ex[q].y * ey.y, xi = ex[q].x * ey.y + ex[q].y * ey.x;
                re[q] = cr * xr - ci * xi;
                im[q] = cr * xi + ci * xr;
            }
            char *pb = (char *)P + (size_t)bg * Pl * ps * es;
            if constexpr (F == FMT_BF16X4) {
                if (sr) {  // BF16x3 form: stochastic split, random bits keyed by the slot-local PSF index
                    store_cplx8_sr(pb, ps, (size_t)ny * ldi + nx0, re, im, ((size_t)(bg - r * B) * ni + ny) * ldi + nx0,
                                   sr ^ 0x1b873593u);
                    continue;
                }
            }
            store_cplx8<F>(pb, ps, (size_t)ny * ldi + nx0, re, im);
        }
    }
}

// The phasor of the mirror-paired forward (FP16 split form; pair_layout in dlx_common.cuh).
// One thread takes a quadrant point jy and QW pair indices jx .. jx+QW-1 for one wavelength: the
// 4 QW samples (jy or Ni-1-jy, jx+q or Ni-1-jx-q) of T_hat exp(i 2 pi OPD / lambda), times the
// tilts of each source and exposure, give (a) the plain phasor P, written as k_phasor writes it
// (pi_r P; the adjoint 1^T epilogue reads it), and (b) the sums and differences along both axes
// into Pp, times pi_r / 4 (a sum of four samples of modulus <= 1 stays <= 1).  A mirror that is
// its own sample (the middle row or column of an odd pupil) counts once: its partner is taken
// as zero.  Grid: x over (jy, group of QW jx), y over (slot, wavelength).
template <int N>
struct HVec;  // N halves stored as one vector
template <>
struct HVec<4> {
    using T = uint2;
};
template <>
struct HVec<2> {
    using T = unsigned int;
};
template <int N>
__device__ __forceinline__ void store_pairN(__half *q, size_t ps, const float (&v1)[N], const float (&v2)[N]) {
    using H = H16<FMT_F16X4>;
    using V = typename HVec<N>::T;
    __align__(8) __half h1[N], l1[N], h2[N], l2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        h1[i] = H::hi(v1[i]);
        l1[i] = H::from(v1[i] - H::to(h1[i]));
        h2[i] = H::hi(v2[i]);
        l2[i] = H::from(v2[i] - H::to(h2[i]));
    }
    *(V *)q = *(const V *)h1;
    *(V *)(q + ps) = *(const V *)l1;
    *(V *)(q + 2 * ps) = *(const V *)h2;
    *(V *)(q + 3 * ps) = *(const V *)l2;
}

// N consecutive elements of a four-plane FP16 split operand (aligned to 2 N bytes): one 2 N-byte
// store per plane.
template <int N>
__device__ __forceinline__ void store_cplxN_f16(__half *p, size_t ps, const float (&re)[N], const float (&im)[N]) {
    using H = H16<FMT_F16X4>;
    using V = typename HVec<N>::T;
    __align__(8) __half rh[N], rl[N], ih[N], il[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        rh[i] = H::hi(re[i]);
        rl[i] = H::from(re[i] - H::to(rh[i]));
        ih[i] = H::hi(im[i]);
        il[i] = H::from(im[i] - H::to(ih[i]));
    }
    *(V *)p = *(const V *)rh;
    *(V *)(p + ps) = *(const V *)rl;
    *(V *)(p + 2 * ps) = *(const V *)ih;
    *(V *)(p + 3 * ps) = *(const V *)il;
}

template <int QW>
__global__ void __launch_bounds__(256, QW == 4 ? 2 : 3) k_phasor_pair(DevParams prm, const float *__restrict__ opd,
                                                     const float2 *__restrict__ tilt, const float *__restrict__ invlam,
                                                     const float *__restrict__ pscale, int B, int nl, int nse, int ne,
                                                     int ni, int ldi, void *P, void *Pp, int hn, int hp, int ldk,
                                                     const float *__restrict__ tmap, float tcoef, uint32_t tmask) {
    pdl_wait();
    constexpr int F = FMT_F16X4;
    const int npx = ni * ni, ng = (hn + QW - 1) / QW;
    const int r = blockIdx.y / nl, l = blockIdx.y - r * nl;
    const float *T = slot_ptr(prm, PT, r), *op = opd + (size_t)r * npx;
    const float sc = pscale[2 * r] * pscale[2 * r + 1], il = invlam[l];
    const size_t ps = (size_t)ni * ldi, pps = (size_t)2 * hp * ldk;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < hn * ng; it += gridDim.x * blockDim.x) {
        const int jy = it / ng, jx0 = QW * (it - jy * ng);
        const int ys[2] = {jy, ni - 1 - jy};
        // T_hat exp(i 2 pi OPD / lambda) and the tangent coefficient at (ys[a], x of (h, q));
        // h = 1 is the mirror column ni - 1 - (jx0 + q)
        float br[2][2][QW], bi[2][2][QW], ta[2][2][QW];
        bool in[2][2][QW];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int q = 0; q < QW; ++q) {
                    const int jx = jx0 + q, x = h ? ni - 1 - jx : jx;
                    in[a][h][q] = jx < hn && !(a == 1 && ys[1] == ys[0]) && !(h == 1 && x == jx);
                    br[a][h][q] = 0.f;
                    bi[a][h][q] = 0.f;
                    ta[a][h][q] = 0.f;
                    if (!in[a][h][q]) continue;
                    const size_t o = (size_t)ys[a] * ni + x;
                    const float tq = __ldg(T + o) * sc;
                    if (tq != 0.f) {
                        float ph = __ldg(op + o) * il;
                        ph -= rintf(ph);
                        float sn, cs;
                        sincospif(2.f * ph, &sn, &cs);
                        br[a][h][q] = tq * cs;
                        bi[a][h][q] = tq * sn;
                    }
                    if (tmap) ta[a][h][q] = tcoef * 6.283185307f * il * __ldg(tmap + o);
                }
        for (int se = 0; se < nse; ++se) {
            const int bg = r * B + l * nse + se;
            const float2 *tx = tilt + (size_t)bg * 2 * ni, *ty = tx + ni;
            const bool tan = tmap && ((tmask >> (se / ne)) & 1u);
            float pr[2][2][QW], pim[2][2][QW];
            char *pb = (char *)P + (size_t)bg * 4 * ps * 2;
            // QW whole pairs of an axis of a multiple of QW samples: the plain phasor goes out as
            // 2 QW-byte vectors (the mirror columns ni-QW-jx0 .. ni-1-jx0 in increasing order)
            const bool vec = (ni % QW) == 0 && jx0 + QW - 1 < hn;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float2 ey = __ldg(ty + ys[a]);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int q = 0; q < QW; ++q) {
                        pr[a][h][q] = 0.f;
                        pim[a][h][q] = 0.f;
                        if (!in[a][h][q]) continue;
                        const int jx = jx0 + q, x = h ? ni - 1 - jx : jx;
                        float cr = br[a][h][q], ci = bi[a][h][q];
                        if (tan) {  // times (1 + i a)
                            const float t = ta[a][h][q], nr = cr - t * ci;
                            ci = ci + t * cr;
                            cr = nr;
                        }
                        const float2 ex = __ldg(tx + x);
                        const float xr = ex.x * ey.x - ex.y * ey.y, xi = ex.x * ey.y + ex.y * ey.x;
                        const float vr = cr * xr - ci * xi, vi = cr * xi + ci * xr;
                        pr[a][h][q] = vr;
                        pim[a][h][q] = vi;
                        // (a) the plain phasor, split as k_phasor splits it
                        if (!vec) store_cplx<F>(pb, ps, (size_t)ys[a] * ldi + x, vr, vi);
                    }
                if (vec) {
                    float r0[QW], i0[QW], r1[QW], i1[QW];
#pragma unroll
                    for (int q = 0; q < QW; ++q) {
                        r0[q] = pr[a][0][q];
                        i0[q] = pim[a][0][q];
                        r1[q] = pr[a][1][QW - 1 - q];
                        i1[q] = pim[a][1][QW - 1 - q];
                    }
                    __half *pr0 = (__half *)pb + (size_t)ys[a] * ldi;
                    store_cplxN_f16<QW>(pr0 + jx0, ps, r0, i0);
                    store_cplxN_f16<QW>(pr0 + (ni - QW - jx0), ps, r1, i1);
                }
            }
            // (b) Q[Ry][Rx]: Ry pairs the rows (S = sum, D = difference), Rx the columns; column
            // block Rx holds (V1, V2) = (Re, Im) for S and (Im, Re) for D
            __half *qb = (__half *)Pp + (size_t)bg * 4 * pps;
#pragma unroll
            for (int ry = 0; ry < 2; ++ry)
#pragma unroll
                for (int rx = 0; rx < 2; ++rx) {
                    float v1[QW], v2[QW];
#pragma unroll
                    for (int q = 0; q < QW; ++q) {
                        const float sy = ry ? -1.f : 1.f, sx = rx ? -1.f : 1.f;
                        const float qr = (pr[0][0][q] + sx * pr[0][1][q]) + sy * (pr[1][0][q] + sx * pr[1][1][q]);
                        const float qi = (pim[0][0][q] + sx * pim[0][1][q]) + sy * (pim[1][0][q] + sx * pim[1][1][q]);
                        v1[q] = 0.25f * (rx ? qi : qr);
                        v2[q] = 0.25f * (rx ? qr : qi);
                    }
                    const int row = ry * hp + jy, col = rx * hp + jx0;
                    store_pairN<QW>(qb + (size_t)row * ldk + col, pps, v1, v2);
                }
        }
    }
}

// columns per thread of the paired phasor: with two (80 registers, three blocks per SM) the
// calibration workload's prologue and phasor build took 0.161 ms, with four (128 registers) 0.174
constexpr int kPhasorQW = 2;
cudaError_t launch_prologue(dlx_plan *p, const DevParams &prm, int R, cudaStream_t st) {
    const int npx = p->ni * p->ni;
    KScope ks(p, KC_PROLOGUE, 2, st);
    const int work = std::max((npx + 255) / 256, (p->B * 2 * p->ni + 255) / 256);
    const int blocks = std::max(1, std::min({work, p->sm_count * 8 / R, kNormParts}));
    cudaError_t e = launch_pdl(k_prologue, dim3(blocks, R), dim3(256), sizeof(float) * (p->nz > 0 ? p->nz : 1), st,
                               prm, p->nz, npx, p->nl, p->opd, p->npart, p->tpart, p->ncount, p->pscale, p->wnorm,
                               p->lam_d, p->B, p->nse, p->ne, p->ni, p->dx, p->tilt, p->qmax, p->gmax, p->chirp);
    if (e != cudaSuccess) return e;
    const int nyl = R * p->nl;
    if (p->paired) {
        const int items = p->hn * ((p->hn + kPhasorQW - 1) / kPhasorQW);
        const int px = std::max(1, std::min((items + 255) / 256, (p->sm_count * 16 + nyl - 1) / nyl));
        return launch_pdl(k_phasor_pair<kPhasorQW>, dim3(px, nyl), dim3(256), 0, st, prm, p->opd, p->tilt, p->invlam, p->pscale,
                          p->B, p->nl, p->nse, p->ne, p->ni, p->ldi, p->P.ptr, p->Pp.ptr, p->hn, p->hp, p->ldk,
                          p->tan_map, p->tan_coef, p->tan_mask);
    }
    const int groups = p->ni * (p->ldi / 8);
    const int px = std::max(1, std::min((groups + 255) / 256, (p->sm_count * 16 + nyl - 1) / nyl));
    DLX_FMT_DISPATCH(p->fmt, F,
                     e = launch_pdl(k_phasor<F>, dim3(px, nyl), dim3(256), 0, st, prm, p->opd, p->tilt, p->invlam,
                                    p->pscale, p->B, p->nl, p->nse, p->ne, p->ni, p->ldi, p->P.ptr, p->sr,
                                    p->tan_map, p->tan_coef, p->tan_mask));
    return e;
}

// ---------------------------------------------------------------------------
// Binning, flat field and Poisson NLL (Sec. 3 pixel response, Sec. 4 likelihood).
// One thread per detector pixel p of slot r = blockIdx.y:
//   B_{e,s}[p] = sum over the os x os block and the partial-intensity planes,
//   m = FF sum_s F_s B_{e,s};  L += m - d ln max(m, 1e-30);
//   g_m = 1 - d / max(m, 1e-30);  GI = FF g_m;  dL/dFF[p] = sum_e g_m B_e;
//   flux partials sum_p FF g_m B_{e,s}.
// Per-block partials (converted to FP64 once) go to red[r][blk][1 + kMaxSrc];
// with data, the last block of the slot to finish sums them in a fixed order into
// loss[r] and dL/dF_s (bcount counts the finished blocks and is reset by it).
// With qmax (FP16 form, loss and gradient) the same pass finds
// Q_{s,e} = max over oversampled pixels q of |GI_e(bin q)| sqrt(I_{s,e}(q)), the
// bound behind the scale of the adjoint field operand; maxima of non-negative
// floats compare as their bit patterns, so the atomic maxima are exact and
// order-independent.
// OS > 0 fixes the oversample at compile time (unrolled, vector loads of the
// os-wide row segments); OS = 0 takes it from `os_rt`.
// Precision (the reading of the target's FP64 loss and gradient reductions): the
// per-pixel loss and flux terms are summed in compensated FP32 pairs (about 44
// significant bits) within a block, each block partial is converted to FP64 once,
// and the last block adds the partials in FP64 in block order.
constexpr int kQShared = 64;  // (source, exposure) maxima kept in shared memory

template <int OS, int MAXS>
__global__ void k_bin_nll(const float *__restrict__ Is, int G, int Rnse, int nse, int ns, int ne, int nd, int os_rt,
                          int no, DevParams prm, const int32_t *__restrict__ data, size_t dstride,
                          float *__restrict__ model, size_t mstride, float *__restrict__ GI, DevGrads g, double *red,
                          unsigned long long *clamped, unsigned int *qmax, double *loss, unsigned int *bcount,
                          float prf_inv, const float *__restrict__ cot, const uint8_t *__restrict__ used, int tn) {
    pdl_wait();
    __shared__ df sh[32 * (1 + MAXS)];
    __shared__ unsigned int s_q[kQShared];
    __shared__ bool s_last;
    const int np = nd * nd, r = blockIdx.y, os = OS > 0 ? OS : os_rt;
    const float *flux = slot_ptr(prm, PFLUX, r), *flat = slot_ptr(prm, PFLAT, r);
    const int32_t *dat = data ? data + (size_t)r * dstride : nullptr;
    float *mod = model + (size_t)r * mstride;
    float *dflat = g.p[GFLAT] ? g.p[GFLAT] + (size_t)r * g.s[GFLAT] : nullptr;
    // with a cotangent the weights dL/dm are cot itself (vector-Jacobian product, no loss)
    const float *ct = cot ? cot + (size_t)r * ne * np : nullptr;
    const bool grad = dat || ct;
    const bool wantq = qmax && grad;
    if (wantq)
        for (int i = threadIdx.x; i < kQShared; i += blockDim.x) s_q[i] = 0u;
    __syncthreads();
    df acc[1 + MAXS];
#pragma unroll
    for (int i = 0; i < 1 + MAXS; ++i) acc[i] = {0.f, 0.f};
    unsigned long long nclamp = 0;
    const size_t plane = (size_t)no * no;
    // block-uniform trip count, so the warp-wide maxima below see every lane
    for (int p0 = blockIdx.x * blockDim.x; p0 < np; p0 += gridDim.x * blockDim.x) {
        const int p = p0 + threadIdx.x;
        const bool valid = p < np;
        const int py = valid ? p / nd : 0, px = valid ? p % nd : 0;
        const float ff = valid ? flat[p] : 0.f;
        float dff = 0.f;
#pragma unroll 2
        for (int e = 0; e < ne; ++e) {
            float bs[MAXS], bmax[MAXS];
            float btot = 0.f;
            const int ry = py * os, rx = px * os;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                bs[s] = 0.f;
                bmax[s] = 0.f;
                if (s < ns && valid) {
                    const size_t rse = (size_t)r * nse + s * ne + e;
                    // planes this block's 128-tile of the intensity holds (os divides 128)
                    const int ng = (used && OS > 0) ? used[rse * tn * tn + (ry >> 7) * tn + (rx >> 7)] : G;
                    float v = 0.f, vm = 0.f;
                    if constexpr (OS == 4 || OS == 2) {
                        // per-subpixel sums over the planes; each plane's OS row loads are in flight together
                        float q[OS][OS];
#pragma unroll
                        for (int a = 0; a < OS; ++a)
#pragma unroll
                            for (int c = 0; c < OS; ++c) q[a][c] = 0.f;
                        for (int gg = 0; gg < ng; ++gg) {
                            const float *src = Is + ((size_t)gg * Rnse + rse) * plane + (size_t)ry * no + rx;
                            if constexpr (OS == 4) {
                                float4 t[4];
#pragma unroll
                                for (int a = 0; a < 4; ++a) t[a] = __ldg((const float4 *)(src + (size_t)a * no));
#pragma unroll
                                for (int a = 0; a < 4; ++a) {
                                    q[a][0] += t[a].x;
                                    q[a][1] += t[a].y;
                                    q[a][2] += t[a].z;
                                    q[a][3] += t[a].w;
                                }
                            } else {
                                const float2 t0 = __ldg((const float2 *)src), t1 = __ldg((const float2 *)(src + no));
                                q[0][0] += t0.x;
                                q[0][1] += t0.y;
                                q[1][0] += t1.x;
                                q[1][1] += t1.y;
                            }
                        }
#pragma unroll
                        for (int a = 0; a < OS; ++a) {
                            float rsum = 0.f;
#pragma unroll
                            for (int c = 0; c < OS; ++c) {
                                rsum += q[a][c];
                                vm = fmaxf(vm, q[a][c]);
                            }
                            v += rsum;
                        }
                    } else {
                        for (int a = 0; a < os; ++a)
                            for (int c = 0; c < os; ++c) {
                                float q = 0.f;
                                const int ngq = used ? used[rse * tn * tn + ((ry + a) >> 7) * tn + ((rx + c) >> 7)] : G;
                                for (int gg = 0; gg < ngq; ++gg)
                                    q += __ldg(Is + ((size_t)gg * Rnse + rse) * plane + (size_t)(ry + a) * no +
                                               (size_t)rx + c);
                                v += q;
                                vm = fmaxf(vm, q);
                            }
                    }
                    bs[s] = v;
                    bmax[s] = vm;
                    btot = fmaf(flux[s], v, btot);
                }
            }
            const float m = ff * btot;
            float gi = 0.f;
            if (valid) {
                mod[(size_t)e * np + p] = m;
                if (grad) {
                    float gm;
                    if (ct) {
                        gm = __ldg(ct + (size_t)e * np + p);
                    } else {
                        const float d = (float)dat[(size_t)e * np + p];
                        float mc = m;
                        if (!(mc >= 1e-30f)) {
                            mc = 1e-30f;
                            ++nclamp;
                        }
                        acc[0] = df_add(acc[0], m);
                        acc[0] = df_add(acc[0], -d * logf(mc));
                        gm = 1.f - d / mc;
                    }
                    gi = ff * gm;
                    GI[((size_t)r * ne + e) * np + p] = gi;
                    dff = fmaf(gm, btot, dff);
#pragma unroll
                    for (int s = 0; s < MAXS; ++s)
                        if (s < ns) acc[1 + s] = df_add(acc[1 + s], gi * bs[s]);
                }
            }
            if (wantq) {
#pragma unroll
                for (int s = 0; s < MAXS; ++s) {
                    if (s >= ns) break;
                    float qv = fabsf(gi) * sqrtf(bmax[s]);
                    if (!(qv < 3.0e38f)) qv = 3.0e38f;  // NaN / inf in the model: keep the bound finite
                    for (int o = 16; o > 0; o >>= 1) qv = fmaxf(qv, __shfl_xor_sync(0xffffffffu, qv, o));
                    if ((threadIdx.x & 31) == 0) {
                        const int k = s * ne + e;
                        if (k < kQShared)
                            atomicMax(s_q + k, __float_as_uint(qv));
                        else
                            atomicMax(qmax + (size_t)r * nse + k, __float_as_uint(qv));
                    }
                }
            }
        }
        if (valid && dat && !ct && prf_inv > 0.f) {
            // chi^2 log prior on the pixel response (Sec. 4): (FF - 1)^2 / (2 sigma^2)
            const float dev = ff - 1.f;
            acc[0] = df_add(acc[0], 0.5f * prf_inv * dev * dev);
            dff = fmaf(prf_inv, dev, dff);
        }
        if (valid && grad && dflat) dflat[p] = dff;
    }
    block_sum<1 + MAXS>(acc, sh);
    if (wantq)
        for (int k = threadIdx.x; k < nse && k < kQShared; k += blockDim.x)
            atomicMax(qmax + (size_t)r * nse + k, s_q[k]);
    if (dat && nclamp) atomicAdd(clamped, nclamp);  // integer count: order-independent
    if (threadIdx.x == 0) {
        for (int i = 0; i < 1 + MAXS; ++i)
            red[((size_t)r * gridDim.x + blockIdx.x) * (1 + kMaxSrc) + i] = df_to_double(acc[i]);
        s_last = false;
        if (grad && bcount) {
            __threadfence();
            s_last = atomicAdd(bcount + r, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (s_last) {
        // loss and dL/dF_s of the slot: one warp per quantity, FP64 over the block partials
        __threadfence();
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = w; i <= ns; i += blockDim.x >> 5) {
            double v = 0.0;
            const double *src = red + (size_t)r * gridDim.x * (1 + kMaxSrc) + i;
            int b = lane;
            for (; b + 96 < (int)gridDim.x; b += 128) {  // four loads in flight
                const double x0 = __ldcg(src + (size_t)b * (1 + kMaxSrc)), x1 = __ldcg(src + (size_t)(b + 32) * (1 + kMaxSrc));
                const double x2 = __ldcg(src + (size_t)(b + 64) * (1 + kMaxSrc)), x3 = __ldcg(src + (size_t)(b + 96) * (1 + kMaxSrc));
                v += x0;
                v += x1;
                v += x2;
                v += x3;
            }
            for (; b < (int)gridDim.x; b += 32) v += __ldcg(src + (size_t)b * (1 + kMaxSrc));
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                if (i == 0) {
                    if (loss) loss[r] = v;
                } else if (g.p[GFLUX]) {
                    g.p[GFLUX][(size_t)r * g.s[GFLUX] + (i - 1)] = (float)v;
                }
            }
        }
        if (threadIdx.x == 0) bcount[r] = 0;  // ready for the next launch
    }
}

// ---------------------------------------------------------------------------
// Many sources (more than 8): the same quantities in two passes, so that no thread
// holds per-source arrays (the one-pass kernel above needs about 7 registers per
// source and drops to one block per SM at 32 sources).
//   k_bin_model:  one thread per pixel; for every image the source loop forms
//                 m = FF sum_s F_s B_s, the NLL, GI = FF g_m and dL/dFF; the loss
//                 partials go to red_a[r][blk] and the slot's last block sums them.
//   k_flux_grad:  grid (blocks, source, slot); dL/dF_s = sum_{e,p} GI_e[p] B_{s,e}[p]
//                 re-reading the source's planes, and the FP16 form's bounds Q_{s,e};
//                 partials in red_b[r][s][blk], the last block of each (r, s) sums them.
// Precision: per-pixel terms are summed in compensated FP32 pairs within a block, block
// partials converted to FP64 once and added in FP64 in block order by the last block.

// For NC oversampled blocks at once (top-left samples src[k] of the first partial-
// intensity plane, skipped where on[k] is false): v[k] = the sum over the os x os block
// and the G planes (gstride floats apart), vm[k] = the largest single oversampled value
// of the block.  The plane loop is outermost and the NC blocks innermost (unrolled), so
// every load of one plane is in flight at once.
template <int OS, int NC>
__device__ __forceinline__ void bin_blocks(const float *const (&src)[NC], int G, size_t gstride, int no, int os,
                                           const bool (&on)[NC], float (&v)[NC], float (&vm)[NC]) {
    if constexpr (OS == 0) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            v[k] = 0.f;
            vm[k] = 0.f;
            if (!on[k]) continue;
            for (int a = 0; a < os; ++a)
                for (int c = 0; c < os; ++c) {
                    float q = 0.f;
                    for (int gg = 0; gg < G; ++gg) q += __ldg(src[k] + gg * gstride + (size_t)a * no + c);
                    v[k] += q;
                    vm[k] = fmaxf(vm[k], q);
                }
        }
    } else {
        float q[NC][OS][OS];
#pragma unroll
        for (int k = 0; k < NC; ++k)
#pragma unroll
            for (int a = 0; a < OS; ++a)
#pragma unroll
                for (int c = 0; c < OS; ++c) q[k][a][c] = 0.f;
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if (!on[k]) continue;
                const float *sp = src[k] + gg * gstride;
                if constexpr (OS == 4) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float4 t = __ldg((const float4 *)(sp + (size_t)a * no));
                        q[k][a][0] += t.x;
                        q[k][a][1] += t.y;
                        q[k][a][2] += t.z;
                        q[k][a][3] += t.w;
                    }
                } else if constexpr (OS == 2) {
                    const float2 t0 = __ldg((const float2 *)sp), t1 = __ldg((const float2 *)(sp + no));
                    q[k][0][0] += t0.x;
                    q[k][0][1] += t0.y;
                    q[k][1][0] += t1.x;
                    q[k][1][1] += t1.y;
                } else {
                    q[k][0][0] += __ldg(sp);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            v[k] = 0.f;
            vm[k] = 0.f;
#pragma unroll
            for (int a = 0; a < OS; ++a) {
                float rsum = 0.f;
#pragma unroll
                for (int c = 0; c < OS; ++c) {
                    rsum += q[k][a][c];
                    vm[k] = fmaxf(vm[k], q[k][a][c]);
                }
                v[k] += rsum;
            }
        }
    }
}

// blocks handled together per thread: fewer for the wide oversampled blocks (registers)
template <int OS>
__host__ __device__ constexpr int bin_chunk() {
    return OS == 4 ? 2 : OS == 2 ? 4 : OS == 1 ? 8 : 1;
}

template <int OS>
__global__ void __launch_bounds__(256) k_bin_model(const float *__restrict__ Is, int G, int Rnse, int nse, int ns,
                                                   int ne, int nd, int os_rt, int no, DevParams prm,
                                                   const int32_t *__restrict__ data, size_t dstride,
                                                   float *__restrict__ model, size_t mstride, float *__restrict__ GI,
                                                   DevGrads g, double *red_a, unsigned long long *clamped,
                                                   double *loss, unsigned int *bcount, float prf_inv,
                                                   const float *__restrict__ cot) {
    pdl_wait();
    __shared__ df sh[32];
    __shared__ float s_flux[kMaxSrc];
    __shared__ bool s_last;
    const int np = nd * nd, r = blockIdx.y, os = OS > 0 ? OS : os_rt;
    const float *flux = slot_ptr(prm, PFLUX, r), *flat = slot_ptr(prm, PFLAT, r);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) s_flux[i] = flux[i];
    __syncthreads();
    const int32_t *dat = data ? data + (size_t)r * dstride : nullptr;
    float *mod = model + (size_t)r * mstride;
    float *dflat = g.p[GFLAT] ? g.p[GFLAT] + (size_t)r * g.s[GFLAT] : nullptr;
    const float *ct = cot ? cot + (size_t)r * ne * np : nullptr;
    const bool grad = dat || ct;
    const size_t plane = (size_t)no * no, gstride = (size_t)Rnse * plane, sstride = (size_t)ne * plane;
    const float *slot = Is + (size_t)r * nse * plane;
    df acc[1] = {{0.f, 0.f}};
    unsigned long long nclamp = 0;
    constexpr int NC = bin_chunk<OS>();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int py = p / nd, px = p % nd;
        const float ff = flat[p];
        float dff = 0.f;
        for (int e = 0; e < ne; ++e) {
            // first source's plane of this exposure, at the block's top-left sample
            const float *base = slot + (size_t)e * plane + (size_t)(py * os) * no + (size_t)px * os;
            float btot = 0.f;
#pragma unroll 1
            for (int s0 = 0; s0 < ns; s0 += NC) {
                const float *src[NC];
                bool on[NC];
                float v[NC], vm[NC];
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    on[k] = s0 + k < ns;
                    src[k] = base + (size_t)(s0 + k) * sstride;
                }
                bin_blocks<OS, NC>(src, G, gstride, no, os, on, v, vm);
#pragma unroll
                for (int k = 0; k < NC; ++k)
                    if (on[k]) btot = fmaf(s_flux[s0 + k], v[k], btot);
            }
            const float m = ff * btot;
            mod[(size_t)e * np + p] = m;
            if (grad) {
                float gm;
                if (ct) {
                    gm = __ldg(ct + (size_t)e * np + p);
                } else {
                    const float d = (float)dat[(size_t)e * np + p];
                    float mc = m;
                    if (!(mc >= 1e-30f)) {
                        mc = 1e-30f;
                        ++nclamp;
                    }
                    acc[0] = df_add(acc[0], m);
                    acc[0] = df_add(acc[0], -d * logf(mc));
                    gm = 1.f - d / mc;
                }
                GI[((size_t)r * ne + e) * np + p] = ff * gm;
                dff = fmaf(gm, btot, dff);
            }
        }
        if (dat && !ct && prf_inv > 0.f) {
            // chi^2 log prior on the pixel response (Sec. 4): (FF - 1)^2 / (2 sigma^2)
            const float dev = ff - 1.f;
            acc[0] = df_add(acc[0], 0.5f * prf_inv * dev * dev);
            dff = fmaf(prf_inv, dev, dff);
        }
        if (grad && dflat) dflat[p] = dff;
    }
    if (!grad) return;
    block_sum<1>(acc, sh);
    if (dat && nclamp) atomicAdd(clamped, nclamp);
    if (threadIdx.x == 0) {
        red_a[(size_t)r * gridDim.x + blockIdx.x] = df_to_double(acc[0]);
        __threadfence();
        s_last = atomicAdd(bcount + r, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        __threadfence();
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += __ldcg(red_a + (size_t)r * gridDim.x + b);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            if (loss) loss[r] = v;
            bcount[r] = 0;  // ready for the next launch
        }
    }
}

template <int OS>
__global__ void __launch_bounds__(256) k_flux_grad(const float *__restrict__ Is, int G, int Rnse, int nse, int ne,
                                                   int nd, int os_rt, int no, const float *__restrict__ GI,
                                                   DevGrads g, double *red_b, unsigned int *fcount,
                                                   unsigned int *qmax) {
    pdl_wait();
    __shared__ df sh[32];
    __shared__ unsigned int s_q[kQShared];
    __shared__ bool s_last;
    const int np = nd * nd, s = blockIdx.y, r = blockIdx.z, os = OS > 0 ? OS : os_rt;
    const size_t plane = (size_t)no * no, gstride = (size_t)Rnse * plane;
    const float *src0 = Is + ((size_t)r * nse + (size_t)s * ne) * plane;  // this source's first plane
    const float *gslot = GI + (size_t)r * ne * np;
    if (qmax)
        for (int i = threadIdx.x; i < kQShared; i += blockDim.x) s_q[i] = 0u;
    __syncthreads();
    df acc[1] = {{0.f, 0.f}};
    constexpr int NC = bin_chunk<OS>();
    // block-uniform trip count, so the warp-wide maxima below see every lane
    for (int p0 = blockIdx.x * blockDim.x; p0 < np; p0 += gridDim.x * blockDim.x) {
        const int p = p0 + threadIdx.x;
        const bool valid = p < np;
        const int py = valid ? p / nd : 0, px = valid ? p % nd : 0;
#pragma unroll 1
        for (int e0 = 0; e0 < ne; e0 += NC) {
            const float *src[NC];
            bool on[NC];
            float v[NC], vm[NC], gi[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const int e = e0 + k;
                on[k] = valid && e < ne;
                src[k] = src0 + (size_t)e * plane + (size_t)(py * os) * no + (size_t)px * os;
                gi[k] = on[k] ? __ldg(gslot + (size_t)e * np + p) : 0.f;
            }
            bin_blocks<OS, NC>(src, G, gstride, no, os, on, v, vm);
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if (e0 + k >= ne) break;
                if (on[k]) acc[0] = df_add(acc[0], gi[k] * v[k]);
                if (qmax) {
                    float qv = fabsf(gi[k]) * sqrtf(vm[k]);
                    if (!(qv < 3.0e38f)) qv = 3.0e38f;  // NaN / inf in the model: keep the bound finite
                    for (int o = 16; o > 0; o >>= 1) qv = fmaxf(qv, __shfl_xor_sync(0xffffffffu, qv, o));
                    if ((threadIdx.x & 31) == 0) {
                        const int e = e0 + k;
                        if (e < kQShared)
                            atomicMax(s_q + e, __float_as_uint(qv));
                        else
                            atomicMax(qmax + (size_t)r * nse + s * ne + e, __float_as_uint(qv));
                    }
                }
            }
        }
    }
    block_sum<1>(acc, sh);  // its barriers also publish s_q
    if (qmax)
        for (int k = threadIdx.x; k < ne && k < kQShared; k += blockDim.x)
            atomicMax(qmax + (size_t)r * nse + s * ne + k, s_q[k]);
    const size_t slot = (size_t)r * kMaxSrc + s;
    if (threadIdx.x == 0) {
        red_b[slot * gridDim.x + blockIdx.x] = df_to_double(acc[0]);
        __threadfence();
        s_last = atomicAdd(fcount + slot, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        __threadfence();
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += __ldcg(red_b + slot * gridDim.x + b);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            if (g.p[GFLUX]) g.p[GFLUX][(size_t)r * g.s[GFLUX] + s] = (float)v;
            fcount[slot] = 0;  // ready for the next launch
        }
    }
}

// ---------------------------------------------------------------------------
// Integer-dither windows.  Every image is a window of the same per-source planes, so
//   k_win_sum:   S[r][P] = sum_s F_s B_s[P] once on the big detector (one thread per pixel);
//   k_win_nll:   m_e[p] = FF[p] S[p + crop[e]], the NLL, GI_e = FF g_m and dL/dFF per image
//                pixel (loss partials as in k_bin_model);
//   k_crop_fold: GI[P] = sum_e GI_e[P - crop[e]] (also the adjoint's weight map);
//   k_win_flux:  dL/dF_s = sum_P GI[P] B_s[P], one pass over each source's plane, and the
//                FP16 form's bound Q_s = max |GI| sqrt(I_s) of the weights the adjoint uses.
// 2-D indexing for the big-detector passes: a thread owns one column px = blockIdx.x *
// blockDim.x + threadIdx.x and walks rows py = blockIdx.y + k * gridDim.y, so no pixel index
// is divided; source (and slot) come from blockIdx.z.  Loss and flux sums: compensated FP32
// pairs within a block, FP64 across block partials in block order (as in k_bin_nll).
template <int OS>
__global__ void __launch_bounds__(128) k_win_sum(const float *__restrict__ Is, int G, int Rnse, int nse, int ns,
                                                 int ndb, int os_rt, int no, DevParams prm, float *__restrict__ S) {
    pdl_wait();
    __shared__ float s_flux[kMaxSrc];
    const int r = blockIdx.z, os = OS > 0 ? OS : os_rt;
    const float *flux = slot_ptr(prm, PFLUX, r);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) s_flux[i] = flux[i];
    __syncthreads();
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= ndb) return;
    const size_t plane = (size_t)no * no, gstride = (size_t)Rnse * plane;
    const float *slot = Is + (size_t)r * nse * plane + (size_t)px * os;
    float *Sr = S + (size_t)r * ndb * ndb + px;
    constexpr int NC = bin_chunk<OS>();
    for (int py = blockIdx.y; py < ndb; py += gridDim.y) {
        const float *base = slot + (size_t)(py * os) * no;
        float btot = 0.f;
#pragma unroll 1
        for (int s0 = 0; s0 < ns; s0 += NC) {
            const float *src[NC];
            bool on[NC];
            float v[NC], vm[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                on[k] = s0 + k < ns;
                src[k] = base + (size_t)(s0 + k) * plane;
            }
            bin_blocks<OS, NC>(src, G, gstride, no, os, on, v, vm);
#pragma unroll
            for (int k = 0; k < NC; ++k)
                if (on[k]) btot = fmaf(s_flux[s0 + k], v[k], btot);
        }
        Sr[(size_t)py * ndb] = btot;
    }
}

__global__ void __launch_bounds__(256) k_win_nll(const float *__restrict__ S, int ndb, int ne, int nd,
                                                 const int2 *__restrict__ crop, DevParams prm,
                                                 const int32_t *__restrict__ data, size_t dstride,
                                                 float *__restrict__ model, size_t mstride, float *__restrict__ GI,
                                                 DevGrads g, double *red_a, unsigned long long *clamped,
                                                 double *loss, unsigned int *bcount, float prf_inv,
                                                 const float *__restrict__ cot) {
    pdl_wait();
    __shared__ df sh[32];
    __shared__ bool s_last;
    const int np = nd * nd, r = blockIdx.y;
    const float *flat = slot_ptr(prm, PFLAT, r), *Sr = S + (size_t)r * ndb * ndb;
    const int32_t *dat = data ? data + (size_t)r * dstride : nullptr;
    float *mod = model + (size_t)r * mstride;
    float *dflat = g.p[GFLAT] ? g.p[GFLAT] + (size_t)r * g.s[GFLAT] : nullptr;
    const float *ct = cot ? cot + (size_t)r * ne * np : nullptr;
    const bool grad = dat || ct;
    df acc[1] = {{0.f, 0.f}};
    unsigned long long nclamp = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int py = p / nd, px = p % nd;
        const float ff = flat[p];
        float dff = 0.f;
        constexpr int EC = 4;  // images per chunk, their loads issued together
        for (int e0 = 0; e0 < ne; e0 += EC) {
            float bt[EC], dv[EC];
#pragma unroll
            for (int k = 0; k < EC; ++k) {
                const int e = e0 + k;
                bt[k] = 0.f;
                dv[k] = 0.f;
                if (e < ne) {
                    const int2 oc = __ldg(crop + e);
                    bt[k] = __ldg(Sr + (size_t)(py + oc.y) * ndb + px + oc.x);
                    if (dat && !ct) dv[k] = (float)__ldg(dat + (size_t)e * np + p);
                }
            }
#pragma unroll
            for (int k = 0; k < EC; ++k) {
                const int e = e0 + k;
                if (e >= ne) break;
                const float btot = bt[k];
                const float m = ff * btot;
                mod[(size_t)e * np + p] = m;
                if (grad) {
                    float gm;
                    if (ct) {
                        gm = __ldg(ct + (size_t)e * np + p);
                    } else {
                        const float d = dv[k];
                        float mc = m;
                        if (!(mc >= 1e-30f)) {
                            mc = 1e-30f;
                            ++nclamp;
                        }
                        acc[0] = df_add(acc[0], m);
                        acc[0] = df_add(acc[0], -d * logf(mc));
                        gm = 1.f - d / mc;
                    }
                    GI[((size_t)r * ne + e) * np + p] = ff * gm;
                    dff = fmaf(gm, btot, dff);
                }
            }
        }
        if (dat && !ct && prf_inv > 0.f) {
            // chi^2 log prior on the pixel response (Sec. 4): (FF - 1)^2 / (2 sigma^2)
            const float dev = ff - 1.f;
            acc[0] = df_add(acc[0], 0.5f * prf_inv * dev * dev);
            dff = fmaf(prf_inv, dev, dff);
        }
        if (grad && dflat) dflat[p] = dff;
    }
    if (!grad) return;
    block_sum<1>(acc, sh);
    if (dat && nclamp) atomicAdd(clamped, nclamp);
    if (threadIdx.x == 0) {
        red_a[(size_t)r * gridDim.x + blockIdx.x] = df_to_double(acc[0]);
        __threadfence();
        s_last = atomicAdd(bcount + r, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        __threadfence();
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += __ldcg(red_a + (size_t)r * gridDim.x + b);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            if (loss) loss[r] = v;
            bcount[r] = 0;  // ready for the next launch
        }
    }
}

template <int OS>
__global__ void __launch_bounds__(128) k_win_flux(const float *__restrict__ Is, int G, int Rnse, int nse, int ns,
                                                  int ndb, int os_rt, int no, const float *__restrict__ GI,
                                                  DevGrads g, double *red_b, unsigned int *fcount,
                                                  unsigned int *qmax) {
    pdl_wait();
    __shared__ df sh[32];
    __shared__ unsigned int s_q;
    __shared__ bool s_last;
    const int s = blockIdx.z % ns, r = blockIdx.z / ns, os = OS > 0 ? OS : os_rt;
    const size_t plane = (size_t)no * no, gstride = (size_t)Rnse * plane;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const bool col = px < ndb;
    const float *src0 = Is + ((size_t)r * nse + s) * plane + (size_t)(col ? px : 0) * os;
    const float *gr = GI + (size_t)r * ndb * ndb + (col ? px : 0);
    if (threadIdx.x == 0) s_q = 0u;
    __syncthreads();
    df acc[1] = {{0.f, 0.f}};
    // NC rows per thread and pass, all their loads in flight; the trip count is the same for
    // every thread of the block, so the warp-wide maxima below see every lane
    constexpr int NC = bin_chunk<OS>();
    for (int py0 = blockIdx.y; py0 < ndb; py0 += gridDim.y * NC) {
        const float *src[NC];
        bool on[NC];
        float v[NC], vm[NC], gi[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const int py = py0 + k * gridDim.y;
            on[k] = col && py < ndb;
            src[k] = src0 + (size_t)((on[k] ? py : 0) * os) * no;
            gi[k] = on[k] ? __ldg(gr + (size_t)py * ndb) : 0.f;
        }
        bin_blocks<OS, NC>(src, G, gstride, no, os, on, v, vm);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (on[k]) acc[0] = df_add(acc[0], gi[k] * v[k]);
            if (qmax) {
                float qv = fabsf(gi[k]) * sqrtf(vm[k]);
                if (!(qv < 3.0e38f)) qv = 3.0e38f;  // NaN / inf in the model: keep the bound finite
                for (int o = 16; o > 0; o >>= 1) qv = fmaxf(qv, __shfl_xor_sync(0xffffffffu, qv, o));
                if ((threadIdx.x & 31) == 0) atomicMax(&s_q, __float_as_uint(qv));
            }
        }
    }
    block_sum<1>(acc, sh);  // its barriers also publish s_q
    if (qmax && threadIdx.x == 0) atomicMax(qmax + (size_t)r * nse + s, s_q);
    const size_t slot = (size_t)r * kMaxSrc + s;
    const int nblk = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        red_b[slot * nblk + bid] = df_to_double(acc[0]);
        __threadfence();
        s_last = atomicAdd(fcount + slot, 1u) == nblk - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        __threadfence();
        double v = 0.0;
        for (int b = threadIdx.x; b < nblk; b += 32) v += __ldcg(red_b + slot * nblk + b);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            if (g.p[GFLUX]) g.p[GFLUX][(size_t)r * g.s[GFLUX] + s] = (float)v;
            fcount[slot] = 0;  // ready for the next launch
        }
    }
}

// Partial-intensity planes of the tensor-core split: the few (slot, source, exposure)
// x 128-tile segments whose wavelengths were cut over several CTAs (fold[i] = (segment,
// planes written)) are added into plane 0 in plane order, so every later reader takes
// plane 0 alone.  Grid: (segments, 16) blocks stepping over the tile's samples.
__global__ void k_plane_fold(float *__restrict__ Is, const int2 *__restrict__ fold, int tn, int no, size_t Rnse) {
    pdl_wait();
    const int2 f = __ldg(fold + blockIdx.x);
    const int tt = tn * tn, rse = f.x / tt, tile = f.x % tt;
    const int m0 = (tile / tn) * 128, n0 = (tile % tn) * 128;
    const int rows = min(128, no - m0), cols = min(128, no - n0);
    const size_t plane = (size_t)no * no;
    float *p0 = Is + (size_t)rse * plane;
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.y * blockDim.x) {
        const size_t o = (size_t)(m0 + i / cols) * no + n0 + i % cols;
        float v = p0[o];
        for (int gg = 1; gg < f.y; ++gg) v += p0[gg * Rnse * plane + o];
        p0[o] = v;
    }
}

cudaError_t launch_plane_fold(dlx_plan *p, int R, cudaStream_t st) {
    if (p->s2.empty() || R < 1 || R > (int)p->s2.size()) return cudaSuccess;
    const dlx_plan::S2Split &sp = p->s2[R - 1];
    if (sp.nfold == 0) return cudaSuccess;
    KScope ks(p, KC_BIN, 1, st);
    return launch_pdl(k_plane_fold, dim3(sp.nfold, 16), dim3(256), 0, st, p->Is, (const int2 *)p->s2_fold + sp.fold,
                      (p->no + 127) / 128, p->no, (size_t)R * p->nse);
}

// GI[r][P] = sum_e GIimg[r][e][P - crop[e]] over the images whose window holds big-detector pixel P
// (fixed order over e)
__global__ void k_crop_fold(const float *__restrict__ gimg, const int2 *__restrict__ crop, int ne, int nd,
                            float *__restrict__ gi, int nb) {
    pdl_wait();
    const int r = blockIdx.y;
    const size_t npb = (size_t)nb * nb, np = (size_t)nd * nd;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < npb; q += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)((unsigned)q / (unsigned)nb), x = (int)((unsigned)q % (unsigned)nb);  // 32-bit division
        float v = 0.f;
        for (int e = 0; e < ne; ++e) {
            const int2 o = __ldg(crop + e);
            const int iy = y - o.y, ix = x - o.x;
            if (iy >= 0 && iy < nd && ix >= 0 && ix < nd) v += __ldg(gimg + ((size_t)r * ne + e) * np + (size_t)iy * nd + ix);
        }
        gi[(size_t)r * npb + q] = v;
    }
}

cudaError_t launch_bin_nll(dlx_plan *p, const DevParams &prm, int R, const int32_t *data, size_t data_stride,
                           float *model, size_t model_stride, const DevGrads *g, double *loss, cudaStream_t st) {
    DevGrads gg{};
    if (g) gg = *g;
    KScope ks(p, KC_BIN, 1, st);
    float *gi = p->GI;
    const int G = planes_to_read(p);
    if (p->crop) {
        // integer-dither windows: one source sum on the big detector, then the images
        const dim3 tb(128);
        const int cx = (p->nd + 127) / 128;
        const int ry = std::max(1, std::min(p->nd, p->sm_count * 16 / (cx * R)));
        auto gs = [&](auto kern) {
            return launch_pdl(kern, dim3(cx, ry, R), tb, 0, st, p->Is, G, R * p->nse, p->nse, p->ns, p->nd, p->os,
                              p->no, prm, p->Swin);
        };
        cudaError_t e = p->os == 4 ? gs(k_win_sum<4>) : p->os == 2 ? gs(k_win_sum<2>) : p->os == 1 ? gs(k_win_sum<1>)
                                                                                                 : gs(k_win_sum<0>);
        ++ks.n;
        if (e == cudaSuccess)
            e = launch_pdl(k_win_nll, dim3(p->bin_a_blocks, R), dim3(256), 0, st, (const float *)p->Swin, p->nd,
                           p->nei, p->ndi, (const int2 *)p->crop, prm, data, data_stride, model, model_stride,
                           p->GIimg, gg, p->red_a, p->clamped, loss, p->bcount, p->prf_inv, p->cot);
        if (e != cudaSuccess || !(data || p->cot)) return e;
        ++ks.n;
        const size_t npb = (size_t)p->nd * p->nd;
        const int bs = (int)std::max<size_t>(1, std::min<size_t>((npb + 255) / 256, (size_t)p->sm_count * 8 / R));
        e = launch_pdl(k_crop_fold, dim3(bs, R), dim3(256), 0, st, (const float *)p->GIimg, (const int2 *)p->crop,
                       p->nei, p->ndi, p->GI, p->nd);
        if (e != cudaSuccess || !(gg.p[GFLUX] || p->qmax)) return e;
        ++ks.n;
        const int fy = win_flux_rows(p, R);
        auto gf = [&](auto kern) {
            return launch_pdl(kern, dim3(cx, fy, p->ns * R), tb, 0, st, p->Is, G, R * p->nse, p->nse, p->ns, p->nd,
                              p->os, p->no, (const float *)p->GI, gg, p->red_b, p->fcount, p->qmax);
        };
        return p->os == 4 ? gf(k_win_flux<4>) : p->os == 2 ? gf(k_win_flux<2>) : p->os == 1 ? gf(k_win_flux<1>)
                                                                                          : gf(k_win_flux<0>);
    }
    auto go = [&](auto kern) {
        // one wave of resident blocks (a grid of several waves left SMs idle in its last one); each
        // block strides over the pixels, so any grid covers them
        static const int per_sm = [&] {
            int n = 0;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, 0) == cudaSuccess && n > 0 ? n : 1;
        }();
        const int blocks = std::max(1, std::min(p->red_blocks, per_sm * p->sm_count / R));
        return launch_pdl(kern, dim3(blocks, R), dim3(256), 0, st, p->Is, G, R * p->nse, p->nse, p->ns,
                          p->ne, p->nd, p->os, p->no, prm, data, data_stride, model,
                          model_stride, gi, gg, p->red, p->clamped, p->qmax, loss, p->bcount, p->prf_inv, p->cot,
                          plane_counts(p, R), (p->no + 127) / 128);
    };
    cudaError_t e;
    if (p->ns <= 8) {
        // one pass, per-source registers (sized for 1, 2 or 8 sources)
        if (p->ns == 1)
            e = p->os == 4 ? go(k_bin_nll<4, 1>) : p->os == 2 ? go(k_bin_nll<2, 1>) : go(k_bin_nll<0, 1>);
        else if (p->ns == 2)
            e = p->os == 4 ? go(k_bin_nll<4, 2>) : p->os == 2 ? go(k_bin_nll<2, 2>) : go(k_bin_nll<0, 2>);
        else
            e = p->os == 4 ? go(k_bin_nll<4, 8>) : p->os == 2 ? go(k_bin_nll<2, 8>) : go(k_bin_nll<0, 8>);
    } else {
        auto ga = [&](auto kern) {
            return launch_pdl(kern, dim3(p->bin_a_blocks, R), dim3(256), 0, st, p->Is, G, R * p->nse, p->nse,
                              p->ns, p->ne, p->nd, p->os, p->no, prm, data,
                              data_stride, model, model_stride, gi, gg, p->red_a, p->clamped, loss, p->bcount,
                              p->prf_inv, p->cot);
        };
        e = p->os == 4 ? ga(k_bin_model<4>) : p->os == 2 ? ga(k_bin_model<2>) : p->os == 1 ? ga(k_bin_model<1>)
                                                                                         : ga(k_bin_model<0>);
        const bool grad = data || p->cot;
        if (e == cudaSuccess && grad && (gg.p[GFLUX] || p->qmax)) {
            ++ks.n;
            auto gb = [&](auto kern) {
                return launch_pdl(kern, dim3(p->bin_b_blocks, p->ns, R), dim3(256), 0, st, p->Is, G,
                                  R * p->nse, p->nse, p->ne, p->nd, p->os, p->no, (const float *)gi, gg, p->red_b,
                                  p->fcount, p->qmax);
            };
            e = p->os == 4 ? gb(k_flux_grad<4>) : p->os == 2 ? gb(k_flux_grad<2>) : p->os == 1 ? gb(k_flux_grad<1>)
                                                                                             : gb(k_flux_grad<0>);
        }
    }
    return e;
}

// psf[e][y][x] = sum_s F_s sum_g Is[g][s nem + em][y + oy][x + ox]: the image-sized oversampled
// intensity of image e (the window at crop[e] of the source's one plane with integer dithers)
__global__ void k_psf_out(const float *__restrict__ Is, int G, int nse, int ns, int nem, int no, int ne, int noi,
                          const int2 *__restrict__ crop, int os, const float *__restrict__ flux, float *__restrict__ psf,
                          const uint8_t *__restrict__ used, int tn) {
    const size_t plane = (size_t)no * no, iplane = (size_t)noi * noi, total = (size_t)ne * iplane;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i / iplane);
        const int y = (int)(i % iplane / noi), x = (int)(i % noi);
        const int2 o = crop ? __ldg(crop + e) : make_int2(0, 0);
        const int em = crop ? 0 : e;
        const int yy = y + o.y * os, xx = x + o.x * os;
        const size_t q = (size_t)yy * no + xx;
        float v = 0.f;
        for (int s = 0; s < ns; ++s) {
            float vs = 0.f;
            const size_t rse = (size_t)s * nem + em;
            const int ng = used ? used[rse * tn * tn + (yy >> 7) * tn + (xx >> 7)] : G;
            for (int gg = 0; gg < ng; ++gg) vs += Is[((size_t)gg * nse + rse) * plane + q];
            v = fmaf(flux[s], vs, v);
        }
        psf[i] = v;
    }
}

cudaError_t launch_psf_out(dlx_plan *p, const DevParams &prm, float *psf, cudaStream_t st) {
    const int noi = p->ndi * p->os;
    const size_t total = (size_t)noi * noi * p->nei;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)p->sm_count * 16);
    KScope ks(p, KC_BIN, 1, st);
    k_psf_out<<<blocks, 256, 0, st>>>(p->Is, planes_to_read(p), p->nse, p->ns, p->ne, p->no, p->nei, noi,
                                      (const int2 *)p->crop, p->os, prm.p[PFLUX], psf, plane_counts(p, 1),
                                      (p->no + 127) / 128);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient reductions.  gphi[bg][n] already carries 2 pi / lambda_l.  Loads are
// issued four or eight at a time ahead of the compensated additions, and long
// sums are split over many blocks, so no kernel waits on one memory latency per
// element.

// g_OPD[r][n] = sum_{b in slot r} gphi[b][n] (compensated);  dL/dOPD_pix = g_OPD;
// and the Zernike partials <Z_j, g_OPD> over the block's 64 pupil pixels
// (zpart[r][j][block], compensated pairs).  A block covers 64 pupil pixels with 4
// threads per pixel, each summing every 4th entry of the pixel's column of gphi (8
// loads in flight); the 4 partial sums are combined in a fixed order.  For the
// Zernike partials the block takes up to 64 terms at a time: their basis rows over
// the block's pixels are staged in shared memory (coalesced 256-byte row loads), each
// thread forms the partial sum of one (term, 8-pixel group) pair, and one thread per
// term adds the term's eight group sums in order.  All sums are compensated FP32 pairs
// (about 44 significant bits), the reading of "FP64 gradient reductions" applied here,
// in a fixed order, so every run gives the same bits.
constexpr int kGopdPx = 64;     // pupil pixels per block of k_gopd_zern
constexpr int kGopdTerms = 64;  // Zernike terms per pass of its partial sums
__global__ void __launch_bounds__(256) k_gopd_zern(const float *__restrict__ gphi, int B, int npx,
                                                   float2 *__restrict__ gopd, DevGrads g, DevParams prm, int nz,
                                                   float2 *__restrict__ zpart) {
    pdl_wait();
    __shared__ df sh[4][kGopdPx];
    __shared__ df ts[kGopdPx];
    __shared__ float zs[kGopdTerms][kGopdPx + 1];  // row stride 65: a warp's terms fall in distinct banks
    __shared__ df part[8 * kGopdTerms];
    const int r = blockIdx.y, px = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const int nb0 = blockIdx.x * kGopdPx, n = nb0 + px;
    df acc{0.f, 0.f};
    if (n < npx) {
        const float *src = gphi + (size_t)r * B * npx + n;
        int b = grp;
        for (; b + 28 < B; b += 32) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __ldg(src + (size_t)(b + 4 * q) * npx);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc = df_add(acc, v[q]);
        }
        for (; b < B; b += 4) acc = df_add(acc, __ldg(src + (size_t)b * npx));
    }
    sh[grp][px] = acc;
    __syncthreads();
    if (grp == 0) {
        const df t = df_add(df_add(sh[0][px], sh[1][px]), df_add(sh[2][px], sh[3][px]));
        ts[px] = t;  // zero beyond the pupil's last pixel
        if (n < npx) {
            gopd[(size_t)r * npx + n] = make_float2(t.hi, t.lo);
            if (g.p[GPIX]) g.p[GPIX][(size_t)r * g.s[GPIX] + n] = t.hi + t.lo;
        }
    }
    if (!zpart) return;
    const float *basis = slot_ptr(prm, PBASIS, r);
    const int nvalid = min(kGopdPx, npx - nb0);
    for (int j0 = 0; j0 < nz; j0 += kGopdTerms) {  // block-uniform
        const int nzc = min(kGopdTerms, nz - j0);
        __syncthreads();  // ts written; zs and part free
        // every thread's basis loads in flight together (blockDim.x = 256: four term rows per pass)
        float zv[kGopdTerms / 4];
#pragma unroll
        for (int k = 0; k < kGopdTerms / 4; ++k) {
            const int jj = 4 * k + (threadIdx.x >> 6), c = threadIdx.x & 63;
            zv[k] = (jj < nzc && c < nvalid) ? __ldg(basis + (size_t)(j0 + jj) * npx + nb0 + c) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kGopdTerms / 4; ++k) {
            const int jj = 4 * k + (threadIdx.x >> 6);
            if (jj < nzc) zs[jj][threadIdx.x & 63] = zv[k];
        }
        __syncthreads();
        // pair i = (term i mod nzc, pixel group i / nzc): sum over the group's 8 pixels
        for (int i = threadIdx.x; i < nzc * 8; i += blockDim.x) {
            const int jj = i % nzc, c0 = 8 * (i / nzc);
            df v{0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float z = zs[jj][c0 + c];
                const df t = ts[c0 + c];
                v = df_add(v, z * t.hi);
                v = df_add(v, z * t.lo);
            }
            part[i] = v;
        }
        __syncthreads();
        if (threadIdx.x < nzc) {
            df w = part[threadIdx.x];
#pragma unroll
            for (int gq = 1; gq < 8; ++gq) w = df_add(w, part[gq * nzc + threadIdx.x]);
            zpart[((size_t)r * nz + j0 + threadIdx.x) * gridDim.x + blockIdx.x] = make_float2(w.hi, w.lo);
        }
    }
}

// Position moments of one PSF entry over the whole pupil: sum_n gphi[e][n] x_n
// and y_n.  One block per entry (PSF x K split), 8 loads in flight per thread.
__global__ void k_pos_moments(const float *__restrict__ gphi, int ni, float dx, double *part) {
    __shared__ df sh[64];
    const int b = blockIdx.x, npx = ni * ni;
    const float cN = 0.5f * (ni - 1);
    const float *src = gphi + (size_t)b * npx;
    df v[2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int n0 = 0; n0 < npx; n0 += 8 * 256) {
        float gv[8];
        int nn[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            nn[q] = n0 + q * 256 + threadIdx.x;
            gv[q] = nn[q] < npx ? __ldg(src + nn[q]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int ny = nn[q] / ni, nx = nn[q] - ny * ni;
            v[0] = df_add(v[0], gv[q] * (((float)nx - cN) * dx));
            v[1] = df_add(v[1], gv[q] * (((float)ny - cN) * dx));
        }
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        part[2 * (size_t)b] = df_to_double(v[0]);
        part[2 * (size_t)b + 1] = df_to_double(v[1]);
    }
}

// dL/dtheta_s = sum over wavelengths, exposures and K splits of the moments of
// source s.  One warp per (slot, source, axis); fixed order.
__global__ void k_pos_final(const double *part, int nsplit, int B, int nl, int ns, int ne, DevGrads g) {
    const int r = blockIdx.x, s = blockIdx.y, ax = blockIdx.z, lane = threadIdx.x;
    const int nt = nl * ne * nsplit;
    double v = 0.0;
    for (int t = lane; t < nt; t += 32) {
        const int sp = t % nsplit, le = t / nsplit;
        const int l = le / ne, e = le % ne;
        const size_t b = (size_t)r * B + (size_t)l * ns * ne + s * ne + e;
        v += part[(b * nsplit + sp) * 2 + ax];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) g.p[GPOS][(size_t)r * g.s[GPOS] + 2 * s + ax] = (float)v;
}

// Final sums of the gradient reductions, grid (n_zern + n_src, R), fixed order, in
// compensated FP32 pairs (the Zernike partials arrive as pairs; about 44 significant bits):
// block j < n_zern: dL/dc_j = sum of the Zernike partials of slot r;
// block n_zern + s (tensor-core forms): dL/dtheta_s from the position moments the
// adjoint 1^T epilogue reduced per (PSF, K split, tile, warp), over wavelengths and
// exposures of source s.
__global__ void k_grad_final(const float2 *__restrict__ zpart, int nz, int nzb, const float *__restrict__ mom,
                             int per_psf, int B, int nl, int ns, int ne, DevGrads g) {
    pdl_wait();
    __shared__ df sh[32 * 2];
    const int r = blockIdx.y, k = blockIdx.x;
    df v[2] = {{0.f, 0.f}, {0.f, 0.f}};
    if (k < nz) {
        const float2 *src = zpart + ((size_t)r * nz + k) * nzb;
        for (int t0 = 0; t0 < nzb; t0 += 4 * blockDim.x) {
            float2 x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int t = t0 + q * blockDim.x + threadIdx.x;
                x[q] = t < nzb ? __ldg(src + t) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) v[0] = df_add(v[0], df{x[q].x, x[q].y});
        }
        block_sum<2>(v, sh);
        if (threadIdx.x == 0) g.p[GZERN][(size_t)r * g.s[GZERN] + k] = v[0].hi + v[0].lo;
    } else {
        const int s = k - nz, nt = nl * ne * per_psf;
        for (int t0 = 0; t0 < nt; t0 += 4 * blockDim.x) {
            float2 x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int t = t0 + q * blockDim.x + threadIdx.x;
                x[q] = make_float2(0.f, 0.f);
                if (t < nt) {
                    const int le = t / per_psf, kk = t - le * per_psf, l = le / ne, e = le - l * ne;
                    const size_t b = (size_t)r * B + (size_t)l * ns * ne + s * ne + e;
                    x[q] = __ldg((const float2 *)mom + b * per_psf + kk);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[0] = df_add(v[0], x[q].x);
                v[1] = df_add(v[1], x[q].y);
            }
        }
        block_sum<2>(v, sh);
        if (threadIdx.x == 0) {
            g.p[GPOS][(size_t)r * g.s[GPOS] + 2 * s] = v[0].hi + v[0].lo;
            g.p[GPOS][(size_t)r * g.s[GPOS] + 2 * s + 1] = v[1].hi + v[1].lo;
        }
    }
}

// The adjoint field from the fields stage 2 kept (the chain rule of the Poisson likelihood,
// Sec. 4, through I = sum_l w_l F_s |E|^2): GEt[z][kx][ky] = 2 w_l F_s GI[e][ky/os][kx/os] E[kx][ky]
// for the chunk-local PSF z = b - b0, b = (r, l, s, e), from Ef (fp32, [b][re, im][kx][ky]) into
// the four-plane 16-bit split, rounded to nearest -- the values and the split that the recomputing
// contraction's epilogue writes.  In the FP16 form Ef holds stage 2's raw accumulators, E times
// alpha_l^2 pi_r sigma1 (and 1/4 when the forward is mirror-paired), and GEt holds gamma_b G_E:
// the row constant takes both scales (the recomputing epilogue's u and gamma), and the pass also
// records max |GEt| of each PSF in gmax for the adjoint 2^T's output scale.  One warp per row
// (z, kx) at a time: the row's constants are formed once, and each lane takes 8-element vectors
// 256 columns apart (two 16-byte loads per plane in, one 16-byte store per plane out, four
// vectors in flight); padding columns ky >= No get zeros.
template <int F>
__device__ __forceinline__ float field_scale_vec(const float *er, const float *ei, typename H16<F>::T *p, size_t ps,
                                                 const float *gi, float c, int k0, int no, int os, int bmax) {
    using H = H16<F>;
    const float4 a0 = __ldg((const float4 *)(er + k0)), a1 = __ldg((const float4 *)(er + k0) + 1);
    const float4 c0 = __ldg((const float4 *)(ei + k0)), c1 = __ldg((const float4 *)(ei + k0) + 1);
    const float xr[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float xi[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    __align__(16) typename H::T rh[8], rl[8], ih[8], il[8];
    int brow = k0 / os, brem = k0 - brow * os;
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool in = k0 + q < no;
        const float f = in ? c * __ldg(gi + min(brow, bmax)) : 0.f;
        const float x = in ? xr[q] * f : 0.f, y = in ? xi[q] * f : 0.f;
        rh[q] = H::hi(x);
        rl[q] = H::from(x - H::to(rh[q]));
        ih[q] = H::hi(y);
        il[q] = H::from(y - H::to(ih[q]));
        if constexpr (F == FMT_F16X4) mx = fmaxf(mx, fmaxf(fabsf(x), fabsf(y)));
        if (++brem == os) {
            brem = 0;
            ++brow;
        }
    }
    *(uint4 *)(p + k0) = *(const uint4 *)rh;
    *(uint4 *)(p + ps + k0) = *(const uint4 *)rl;
    *(uint4 *)(p + 2 * ps + k0) = *(const uint4 *)ih;
    *(uint4 *)(p + 3 * ps + k0) = *(const uint4 *)il;
    return mx;
}

// The same eight columns for the TF32 split form: FP32 planes, hi = the 8-bit split and lo its
// remainder rounded to TF32, as the recomputing epilogue writes them.
__device__ __forceinline__ float field_scale_vec_tf32(const float *er, const float *ei, float *p, size_t ps,
                                                      const float *gi, float c, int k0, int no, int os, int bmax) {
    const float4 a0 = __ldg((const float4 *)(er + k0)), a1 = __ldg((const float4 *)(er + k0) + 1);
    const float4 c0 = __ldg((const float4 *)(ei + k0)), c1 = __ldg((const float4 *)(ei + k0) + 1);
    const float xr[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float xi[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    __align__(16) float rh[8], rl[8], ih[8], il[8];
    int brow = k0 / os, brem = k0 - brow * os;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool in = k0 + q < no;
        const float f = in ? c * __ldg(gi + min(brow, bmax)) : 0.f;
        const float x = in ? xr[q] * f : 0.f, y = in ? xi[q] * f : 0.f;
        rh[q] = split_hi8(x);
        rl[q] = tf32_round(x - rh[q]);
        ih[q] = split_hi8(y);
        il[q] = tf32_round(y - ih[q]);
        if (++brem == os) {
            brem = 0;
            ++brow;
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        *(float4 *)(p + k0 + 4 * h) = *(const float4 *)(rh + 4 * h);
        *(float4 *)(p + ps + k0 + 4 * h) = *(const float4 *)(rl + 4 * h);
        *(float4 *)(p + 2 * ps + k0 + 4 * h) = *(const float4 *)(ih + 4 * h);
        *(float4 *)(p + 3 * ps + k0 + 4 * h) = *(const float4 *)(il + 4 * h);
    }
    return 0.f;
}

template <int F>
using FieldOpT = std::conditional_t<F == FMT_TF32X4, float, typename H16<F>::T>;

template <int F>
__global__ void __launch_bounds__(256) k_field_scale(const float *__restrict__ Ef, FieldOpT<F> *__restrict__ ge,
                                                     const float *__restrict__ GIt, DevParams prm,
                                                     const float *__restrict__ wnorm, int b0, int nb, int B, int nl,
                                                     int nse, int ne, int no, int ldo, int nd, int os,
                                                     const unsigned int *__restrict__ qmax,
                                                     const float *__restrict__ ascale, const float *__restrict__ pscale,
                                                     float sig1, float pf, unsigned int *gmax) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5, nrows = nb * no;
    const size_t ps = (size_t)no * ldo;
    const int bmax = (no - 1) / os;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nrows; row += nwarps) {
        const int z = row / no, kx = row - z * no, b = b0 + z;
        const int r = b / B, rem = b - r * B, l = rem / nse, se = rem - l * nse, s = se / ne, e = se - s * ne;
        const float w = __ldg(wnorm + r * nl + l), fl = __ldg(slot_ptr(prm, PFLUX, r) + s);
        float c = 2.f * w * fl;
        if constexpr (F == FMT_F16X4) {
            // gamma_b = 2^-ceil(log2(2 |F_s| sqrt(w_l) Q_se)) and u = pf / (alpha_l^2 pi_r sigma1)
            const float Q = __uint_as_float(__ldg(qmax + (size_t)r * nse + se));
            const float al = __ldg(ascale + l), pi = __ldg(pscale + 2 * r + 1);
            c *= inv_pow2_ceil(2.f * fabsf(fl) * sqrtf(fabsf(w)) * Q) * (pf / (al * al * pi * sig1));
        }
        const float *gi = GIt + (((size_t)r * ne + e) * nd + kx / os) * nd;  // row x = kx / os, along y
        const float *er = Ef + (size_t)b * 2 * ps + (size_t)kx * ldo, *ei = er + ps;
        FieldOpT<F> *p = ge + (size_t)z * 4 * ps + (size_t)kx * ldo;
        auto vec8 = [&](int k) {
            if constexpr (F == FMT_TF32X4) return field_scale_vec_tf32(er, ei, p, ps, gi, c, k, no, os, bmax);
            else return field_scale_vec<F>(er, ei, p, ps, gi, c, k, no, os, bmax);
        };
        float mx = 0.f;
        int k0 = 8 * lane;
        for (; k0 + 3 * 256 < ldo; k0 += 4 * 256) {
#pragma unroll
            for (int u = 0; u < 4; ++u) mx = fmaxf(mx, vec8(k0 + u * 256));
        }
        for (; k0 < ldo; k0 += 256) mx = fmaxf(mx, vec8(k0));
        if constexpr (F == FMT_F16X4) {
            // max |GEt| of the PSF (non-negative floats order as their bits)
            if (!(mx < 3.0e38f)) mx = 3.0e38f;
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) atomicMax(gmax + b, __float_as_uint(mx));
        }
    }
}

// The same pass for the mirror-paired adjoint (FP16 form; pair_layout in dlx_common.cuh): one
// warp takes the rows jx and No-1-jx of a PSF, each lane four pair indices jy at a time (128 per
// warp and step); the four values G_E at (jx or No-1-jx, jy or No-1-jy) give the sums and
// differences along kx (the row block Rx of GEt, for the adjoint 1^T) and along ky (the column
// block Ry, the adjoint 2^T's contraction), times gamma_b / 4, stored as (V1, V2) = (Re, Im) for
// Ry = S and (Im, Re) for D.  A mirror that is its own row or column (the middle of an odd axis)
// counts once.
__device__ __forceinline__ void load4(const float *p, int c0, bool vec, int n, float (&v)[4]) {
    if (vec) {
        const float4 a = __ldg((const float4 *)(p + c0));
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (c0 + q >= 0 && c0 + q < n) ? __ldg(p + c0 + q) : 0.f;
    }
}

__global__ void __launch_bounds__(256, 3) k_field_scale_pair(const float *__restrict__ Ef, __half *__restrict__ ge,
                                                             const float *__restrict__ GIt, DevParams prm,
                                                             const float *__restrict__ wnorm, int b0, int nb, int B,
                                                             int nl, int nse, int ne, int no, int ldo, int nd, int os,
                                                             int hno, int hpo, int ldko,
                                                             const unsigned int *__restrict__ qmax,
                                                             const float *__restrict__ ascale,
                                                             const float *__restrict__ pscale, float sig1, float pf,
                                                             unsigned int *gmax) {
    using H = H16<FMT_F16X4>;
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5, nrows = nb * hno;
    const size_t ps = (size_t)no * ldo, pps = (size_t)2 * hpo * ldko;
    const int bmax = (no - 1) / os;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nrows; row += nwarps) {
        const int z = row / hno, jx = row - z * hno, b = b0 + z;
        const int r = b / B, rem = b - r * B, l = rem / nse, se = rem - l * nse, s = se / ne, e = se - s * ne;
        const float w = __ldg(wnorm + r * nl + l), fl = __ldg(slot_ptr(prm, PFLUX, r) + s);
        const float Q = __uint_as_float(__ldg(qmax + (size_t)r * nse + se));
        const float al = __ldg(ascale + l), pi = __ldg(pscale + 2 * r + 1);
        // 2 w F, gamma_b, u, and 1/4 for the sums of four values
        const float c = 0.25f * 2.f * w * fl * inv_pow2_ceil(2.f * fabsf(fl) * sqrtf(fabsf(w)) * Q) *
                        (pf / (al * al * pi * sig1));
        const int kx1 = no - 1 - jx;
        const bool row1 = kx1 != jx;
        const float *gi0 = GIt + (((size_t)r * ne + e) * nd + jx / os) * nd;
        const float *gi1 = GIt + (((size_t)r * ne + e) * nd + kx1 / os) * nd;
        const float *er0 = Ef + (size_t)b * 2 * ps + (size_t)jx * ldo, *ei0 = er0 + ps;
        const float *er1 = Ef + (size_t)b * 2 * ps + (size_t)kx1 * ldo, *ei1 = er1 + ps;
        __half *gz = ge + (size_t)z * 4 * pps;
        float mx = 0.f;
        for (int j0 = 4 * lane; j0 < hpo; j0 += 128) {
            const bool vec = (no & 3) == 0 && j0 + 4 <= no;
            // row a, direct columns j0 + q (x) and mirror columns no - 1 - j0 - q (y, reversed below)
            float xr0[4], xi0[4], yr0[4], yi0[4], xr1[4], xi1[4], yr1[4], yi1[4];
            load4(er0, j0, vec, no, xr0);
            load4(ei0, j0, vec, no, xi0);
            load4(er0, no - 4 - j0, vec, no, yr0);
            load4(ei0, no - 4 - j0, vec, no, yi0);
            load4(er1, j0, vec, no, xr1);
            load4(ei1, j0, vec, no, xi1);
            load4(er1, no - 4 - j0, vec, no, yr1);
            load4(ei1, no - 4 - j0, vec, no, yi1);
            // g[a][h]: G_E of row a at the direct (h = 0) and mirror (h = 1) column of pair q
            float g00r[4], g00i[4], g01r[4], g01i[4], g10r[4], g10i[4], g11r[4], g11i[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jy = j0 + q, my = no - 1 - jy;
                const bool in0 = jy < hno, in1 = in0 && my != jy;
                const int c0 = min(jy / os, bmax), c1 = min(my / os, bmax);
                const float f00 = in0 ? c * __ldg(gi0 + c0) : 0.f, f01 = in1 ? c * __ldg(gi0 + c1) : 0.f;
                const float f10 = (in0 && row1) ? c * __ldg(gi1 + c0) : 0.f;
                const float f11 = (in1 && row1) ? c * __ldg(gi1 + c1) : 0.f;
                g00r[q] = f00 * xr0[q];
                g00i[q] = f00 * xi0[q];
                g01r[q] = f01 * yr0[3 - q];
                g01i[q] = f01 * yi0[3 - q];
                g10r[q] = f10 * xr1[q];
                g10i[q] = f10 * xi1[q];
                g11r[q] = f11 * yr1[3 - q];
                g11i[q] = f11 * yi1[3 - q];
            }
#pragma unroll
            for (int rx = 0; rx < 2; ++rx)
#pragma unroll
                for (int ry = 0; ry < 2; ++ry) {
                    const float sx = rx ? -1.f : 1.f, sy = ry ? -1.f : 1.f;
                    __align__(8) __half h1[4], l1[4], h2[4], l2[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float qr = (g00r[q] + sy * g01r[q]) + sx * (g10r[q] + sy * g11r[q]);
                        const float qi = (g00i[q] + sy * g01i[q]) + sx * (g10i[q] + sy * g11i[q]);
                        const float v1 = ry ? qi : qr, v2 = ry ? qr : qi;
                        mx = fmaxf(mx, fmaxf(fabsf(v1), fabsf(v2)));
                        h1[q] = H::hi(v1);
                        l1[q] = H::from(v1 - H::to(h1[q]));
                        h2[q] = H::hi(v2);
                        l2[q] = H::from(v2 - H::to(h2[q]));
                    }
                    __half *o = gz + (size_t)(rx * hpo + jx) * ldko + ry * hpo + j0;
                    *(uint2 *)o = *(const uint2 *)h1;
                    *(uint2 *)(o + pps) = *(const uint2 *)l1;
                    *(uint2 *)(o + 2 * pps) = *(const uint2 *)h2;
                    *(uint2 *)(o + 3 * pps) = *(const uint2 *)l2;
                }
        }
        // max |GEt| of the PSF (non-negative floats order as their bits)
        if (!(mx < 3.0e38f)) mx = 3.0e38f;
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(gmax + b, __float_as_uint(mx));
    }
}

// GIt[k][x][y] = GI[k][y][x] for the R * ne weight maps, through 32 x 32 tiles in shared memory
// (the field scaling reads the weights along y).
__global__ void k_gi_transpose(const float *__restrict__ GI, float *__restrict__ GIt, int nd) {
    __shared__ float t[32][33];
    pdl_wait();
    const size_t base = (size_t)blockIdx.z * nd * nd;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        if (y < nd && x < nd) t[j][threadIdx.x] = GI[base + (size_t)y * nd + x];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int x = x0 + j, y = y0 + threadIdx.x;
        if (y < nd && x < nd) GIt[base + (size_t)x * nd + y] = t[threadIdx.x][j];
    }
}

cudaError_t launch_field_scale(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    KScope ks(p, KC_FIELD_SCALE, 2, st);
    const int R = (b0 + nb + p->B - 1) / p->B;  // slots whose weight maps the PSFs use
    const int tiles = (p->nd + 31) / 32;
    cudaError_t e = launch_pdl(k_gi_transpose, dim3(tiles, tiles, R * p->ne), dim3(32, 8), 0, st,
                               (const float *)p->GI, p->GIt, p->nd);
    if (e != cudaSuccess) return e;
    const int rows = nb * p->no;
    const int blocks = std::max(1, std::min((rows + 7) / 8, p->sm_count * 8));
    auto go = [&](auto kern, void *ge) {
        return launch_pdl(kern, dim3(blocks), dim3(256), 0, st, (const float *)p->Ef, ge, (const float *)p->GIt,
                          prm, (const float *)p->wnorm, b0, nb, p->B, p->nl, p->nse, p->ne, p->no, p->ldo, p->nd,
                          p->os, (const unsigned int *)p->qmax, (const float *)p->ascale, (const float *)p->pscale,
                          inv_pow2_ceil((float)p->ni), p->paired ? 4.f : 1.f, p->gmax);
    };
    if (p->padj) {
        const int prow = nb * p->hno;
        const int pblocks = std::max(1, std::min((prow + 7) / 8, p->sm_count * 8));
        return launch_pdl(k_field_scale_pair, dim3(pblocks), dim3(256), 0, st, (const float *)p->Ef,
                          (__half *)p->GEt.ptr, (const float *)p->GIt, prm, (const float *)p->wnorm, b0, nb, p->B,
                          p->nl, p->nse, p->ne, p->no, p->ldo, p->nd, p->os, p->hno, p->hpo, p->ldko,
                          (const unsigned int *)p->qmax, (const float *)p->ascale, (const float *)p->pscale,
                          inv_pow2_ceil((float)p->ni), p->paired ? 4.f : 1.f, p->gmax);
    }
    if (p->fmt == FMT_F16X4) return go(k_field_scale<FMT_F16X4>, p->GEt.ptr);
    if (p->fmt == FMT_TF32X4) return go(k_field_scale<FMT_TF32X4>, p->GEt.ptr);
    return go(k_field_scale<FMT_BF16X4>, p->GEt.ptr);
}

cudaError_t launch_grad_reduce(dlx_plan *p, const DevParams &prm, int R, const DevGrads *g, cudaStream_t st) {
    const int npx = p->ni * p->ni, nzb = (npx + kGopdPx - 1) / kGopdPx;
    DevGrads gg{};
    if (g) gg = *g;
    const bool zern = gg.p[GZERN] && p->nz > 0, pos_tc = gg.p[GPOS] && p->mom, pos_simt = gg.p[GPOS] && !p->mom;
    const int nfinal = (zern ? p->nz : 0) + (pos_tc ? p->ns : 0);
    KScope ks(p, KC_GRAD, 1 + (nfinal > 0 ? 1 : 0) + (pos_simt ? 2 : 0), st);
    // gphi holds gsplit partial planes per PSF; they are summed with the PSFs
    cudaError_t e = launch_pdl(k_gopd_zern, dim3(nzb, R), dim3(256), 0, st, p->gphi, p->B * p->gsplit, npx, p->gopd,
                               gg, prm, zern ? p->nz : 0, zern ? p->zpart : nullptr);
    if (e != cudaSuccess) return e;
    if (pos_simt) {
        k_pos_moments<<<R * p->B * p->gsplit, 256, 0, st>>>(p->gphi, p->ni, (float)p->dx, p->pos_part);
        k_pos_final<<<dim3(R, p->ns, 2), 32, 0, st>>>(p->pos_part, p->gsplit, p->B, p->nl, p->ns, p->ne, gg);
    }
    if (nfinal > 0) {
        const int tiles = ((p->ni + 127) / 128) * ((p->ni + 127) / 128);
        // source blocks follow the Zernike blocks; with no Zernike gradient they start at 0
        e = launch_pdl(k_grad_final, dim3(nfinal, R), dim3(256), 0, st, p->zpart, zern ? p->nz : 0, nzb, p->mom,
                       p->gsplit * tiles * 8, p->B, p->nl, p->ns, p->ne, gg);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba 2014), the optimiser of Sec. 4.
__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t launch_adam(float *theta, const float *grad, float *m, float *v, size_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_adam<<<blocks, 256, 0, st>>>(theta, grad, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// cot = dL/dm of the Poisson NLL sum (m - d ln m): 1 - d / max(m, 1e-30)
__global__ void k_nll_cotangent(const float *__restrict__ m, const int32_t *__restrict__ d, size_t n,
                                float *__restrict__ cot) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        cot[i] = 1.f - (float)d[i] / fmaxf(m[i], 1e-30f);
}

cudaError_t launch_nll_cotangent(const float *m, const int32_t *d, size_t n, float *cot, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_nll_cotangent<<<blocks, 256, 0, st>>>(m, d, n, cot);
    return cudaGetLastError();
}

// jvp = (m(+alpha) - m(-alpha)) * c, in place over the first operand
__global__ void k_scaled_diff(float *__restrict__ a, const float *__restrict__ b, size_t n, float c) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] = (a[i] - b[i]) * c;
}

cudaError_t launch_scaled_diff(float *a, const float *b, size_t n, float c, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_scaled_diff<<<blocks, 256, 0, st>>>(a, b, n, c);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weighted Gram matrix of the Jacobian rows (Fisher information of the Poisson
// likelihood, Sec. 4): F[i][j] = sum_p J[i][p] J[j][p] w_p over the upper
// triangle.  Each block takes 32-pixel chunks (rows padded to 33 floats so the
// threads of a warp, which share i and run over consecutive j, hit distinct
// banks), sums a chunk in FP32 and adds it to its FP64 partials; a second kernel
// adds the block partials in block order, so the result does not depend on timing
// (FP32 over 32 products, FP64 beyond).
constexpr int kGramChunk = 32, kGramPad = 33, kGramPairsPerThread = (DLX_GRAM_MAX_PAR * (DLX_GRAM_MAX_PAR + 1) / 2 + 255) / 256;

__global__ void __launch_bounds__(256) k_fisher_gram(const float *__restrict__ J, int n, size_t npix,
                                                     const float *__restrict__ model,
                                                     const int32_t *__restrict__ data, double *__restrict__ part) {
    extern __shared__ float sm[];
    float *Js = sm, *Jw = sm + (size_t)n * kGramPad, *w = Jw + (size_t)n * kGramPad;
    const int npair = n * (n + 1) / 2;
    // this thread's pairs k = tid + 256 m, row-major over the upper triangle
    int pij[kGramPairsPerThread];  // i << 8 | j
    double acc[kGramPairsPerThread];
#pragma unroll
    for (int m = 0; m < kGramPairsPerThread; ++m) {
        int k = threadIdx.x + 256 * m, i = 0;
        acc[m] = 0.0;
        if (k < npair) {
            while (k >= n - i) {
                k -= n - i;
                ++i;
            }
        } else {
            k = 0;
        }
        pij[m] = i << 8 | (i + k);
    }
    const size_t nchunk = (npix + kGramChunk - 1) / kGramChunk;
    for (size_t c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const size_t p0 = c * kGramChunk;
        __syncthreads();
        if (threadIdx.x < kGramChunk) {
            const size_t q = p0 + threadIdx.x;
            float wq = 0.f;
            if (q < npix) {
                const float m = fmaxf(model[q], 1e-30f);
                wq = data ? (float)data[q] / (m * m) : 1.f / m;
            }
            w[threadIdx.x] = wq;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * kGramChunk; idx += blockDim.x) {
            const int i = idx / kGramChunk, q = idx % kGramChunk;
            const float v = p0 + q < npix ? __ldg(J + (size_t)i * npix + p0 + q) : 0.f;
            Js[i * kGramPad + q] = v;
            Jw[i * kGramPad + q] = v * w[q];
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kGramPairsPerThread; ++m) {
            if (threadIdx.x + 256 * m >= npair) break;
            const float *a = Jw + (pij[m] >> 8) * kGramPad, *b = Js + (pij[m] & 255) * kGramPad;
            float s = 0.f;
#pragma unroll 8
            for (int q = 0; q < kGramChunk; ++q) s = fmaf(a[q], b[q], s);
            acc[m] += (double)s;
        }
    }
#pragma unroll
    for (int m = 0; m < kGramPairsPerThread; ++m) {
        const int k = threadIdx.x + 256 * m;
        if (k < npair) part[(size_t)blockIdx.x * npair + k] = acc[m];
    }
}

__global__ void k_fisher_final(const double *__restrict__ part, int nb, int n, double *__restrict__ F) {
    const int npair = n * (n + 1) / 2;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npair; k += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < nb; ++b) v += part[(size_t)b * npair + k];
        int i = 0, kk = k;
        while (kk >= n - i) {
            kk -= n - i;
            ++i;
        }
        const int j = i + kk;
        F[(size_t)i * n + j] = v;
        F[(size_t)j * n + i] = v;
    }
}

cudaError_t launch_fisher_gram(const float *J, int n, size_t npix, const float *model, const int32_t *data, double *F,
                               double *work, cudaStream_t st) {
    const size_t nchunk = (npix + kGramChunk - 1) / kGramChunk;
    const int nb = (int)std::min<size_t>(nchunk, DLX_GRAM_BLOCKS);
    const size_t smem = ((size_t)2 * n * kGramPad + kGramChunk) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_fisher_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fisher_gram<<<nb, 256, smem, st>>>(J, n, npix, model, data, work);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int npair = n * (n + 1) / 2;
    k_fisher_final<<<(npair + 255) / 256, 256, 0, st>>>(work, nb, n, F);
    return cudaGetLastError();
}

// Adam over packed slots: element i of slot r belongs to group k with
// off[k] <= i < off[k+1]; a zero learning rate freezes the group.
__global__ void k_adam_slots(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                             float *__restrict__ v, size_t n, int R, const int *__restrict__ off,
                             const float *__restrict__ lr, const int *__restrict__ step, float b1, float b2,
                             float eps) {
    const size_t total = (size_t)R * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / n);
        const int j = (int)(i % n);
        int k = 0;
        while (k < 4 && j >= off[k + 1]) ++k;
        const float a = lr[r * 5 + k];
        if (a == 0.f) continue;
        const int t = step[r];
        const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= a * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t launch_adam_slots(float *theta, const float *grad, float *m, float *v, size_t n, int R, const int *off,
                              const float *lr, const int *step, float b1, float b2, float eps, cudaStream_t st) {
    if (n == 0 || R == 0) return cudaSuccess;
    int blocks = (int)std::min<size_t>(((size_t)R * n + 255) / 256, 8192);
    k_adam_slots<<<blocks, 256, 0, st>>>(theta, grad, m, v, n, R, off, lr, step, b1, b2, eps);
    return cudaGetLastError();
}

}  // namespace dlx
