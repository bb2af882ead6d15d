// Internal declarations of the dlx CUDA library (sm_103a).
//
// Operand layout.  Every complex matrix that feeds a contraction is stored as
// P planes of a row-major [rows][ld] array, plane-major, where ld is the
// contraction length rounded up to a multiple of 64 (operand_ld: the 64-byte row
// chunks the tensor-memory-access engine reads stay aligned; padding columns stay
// zero).  The planes depend
// on the arithmetic form:
//   FMT_F32    : re, im                     (float)         -- CUDA-core FP32 form
//   FMT_BF16X4 : re_hi, re_lo, im_hi, im_lo (bf16)          -- BF16x3 and BF16x4 forms
//   FMT_BF16X2 : re, im                     (bf16)          -- plain BF16 form
//   FMT_TF32X4 : re_hi, re_lo, im_hi, im_lo (tf32 in fp32)  -- TF32x3 form
//   FMT_F16X4  : re_hi, re_lo, im_hi, im_lo (fp16)          -- FP16x3 form
// hi = x rounded to 8 significant bits, lo = x - hi rounded to the element type
// (8 significant bits in BF16, 11 in FP16 and TF32; see split_hi8).  Which split
// products a contraction forms (three, or four with lo*lo) is chosen by the
// tensor-core kernel per form.
// FP16 operands hold x times a power of two that keeps |x| <= 1 (see the
// scale helpers below), so hi and lo stay inside FP16's exponent range.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/dlx.h"

namespace dlx {

enum Fmt { FMT_F32 = 0, FMT_BF16X4 = 1, FMT_BF16X2 = 2, FMT_TF32X4 = 3, FMT_F16X4 = 4 };

__host__ __device__ constexpr int fmt_planes(int f) {
    return (f == FMT_BF16X4 || f == FMT_TF32X4 || f == FMT_F16X4) ? 4 : 2;
}
__host__ __device__ constexpr int fmt_esize(int f) {
    return (f == FMT_BF16X4 || f == FMT_BF16X2 || f == FMT_F16X4) ? 2 : 4;
}

// The hi part of every split keeps 8 significant bits (round to nearest), whatever
// the element type.  The tensor core adds an instruction's products to its FP32
// accumulator after aligning them to it and keeps about 24 bits, truncating: a
// 16-bit hi*hi product (8 x 8 bits) loses nothing beside a sum up to 2^8 times its
// size, whereas the 22-bit products of 11-bit parts (FP16, TF32) lose low bits as
// soon as the sum is 4 times larger, and at a coherent PSF peak those losses add
// up (measured 1.5-1.9e-5 of the peak over a 512-long contraction with full-width
// FP16 and TF32 hi parts).  With an 8-bit hi the lo part of FP16 and TF32 carries
// the next 11 bits, so hi + lo represent x to about 2^-21 (BF16: 2^-17).
__device__ __forceinline__ float split_hi8(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// 16-bit element type of a 16-bit form and its round-to-nearest conversions;
// `hi` rounds the hi part of a split.
template <int F>
struct H16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ T hi(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __bfloat162float(x); }
};
template <>
struct H16<FMT_F16X4> {
    using T = __half;
    static __device__ __forceinline__ T from(float x) { return __float2half_rn(x); }
    // 8 significant bits are exact in FP16 inside its normal range (operands are scaled to |x| <= 1)
    static __device__ __forceinline__ T hi(float x) { return __float2half_rn(split_hi8(x)); }
    static __device__ __forceinline__ float to(T x) { return __half2float(x); }
};

inline int fmt_of_prec(int prec) {
    switch (prec) {
        case DLX_FP32_SIMT: return FMT_F32;
        case DLX_TF32X3: return FMT_TF32X4;
        case DLX_BF16X3: return FMT_BF16X4;
        case DLX_BF16X4: return FMT_BF16X4;
        case DLX_F16X3: return FMT_F16X4;
        case DLX_BF16X3SA: return FMT_BF16X4;
        default: return FMT_BF16X2;
    }
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Store one complex value at element `idx` of a plane-major operand whose
// planes are `pstride` elements apart.
template <int F>
__device__ __forceinline__ void store_cplx(void *base, size_t pstride, size_t idx, float re, float im) {
    if constexpr (F == FMT_F32) {
        float *p = (float *)base;
        p[idx] = re;
        p[pstride + idx] = im;
    } else if constexpr (F == FMT_BF16X4 || F == FMT_F16X4) {
        using H = H16<F>;
        typename H::T *p = (typename H::T *)base;
        const typename H::T rh = H::hi(re), ih = H::hi(im);
        p[idx] = rh;
        p[pstride + idx] = H::from(re - H::to(rh));
        p[2 * pstride + idx] = ih;
        p[3 * pstride + idx] = H::from(im - H::to(ih));
    } else if constexpr (F == FMT_BF16X2) {
        __nv_bfloat16 *p = (__nv_bfloat16 *)base;
        p[idx] = __float2bfloat16_rn(re);
        p[pstride + idx] = __float2bfloat16_rn(im);
    } else {
        float *p = (float *)base;
        float rh = split_hi8(re), ih = split_hi8(im);
        p[idx] = rh;
        p[pstride + idx] = tf32_round(re - rh);
        p[2 * pstride + idx] = ih;
        p[3 * pstride + idx] = tf32_round(im - ih);
    }
}

// Store eight consecutive complex values at element `idx` (a multiple of 8) of
// a plane-major operand: one 16-byte (bf16) or two (fp32) stores per plane.
template <int F>
__device__ __forceinline__ void store_cplx8(void *base, size_t pstride, size_t idx, const float (&re)[8],
                                            const float (&im)[8]) {
    if constexpr (F == FMT_F32 || F == FMT_TF32X4) {
        float *p = (float *)base + idx;
        float hr[8], hi[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            hr[q] = (F == FMT_F32) ? re[q] : split_hi8(re[q]);
            hi[q] = (F == FMT_F32) ? im[q] : split_hi8(im[q]);
        }
        auto put = [&](float *d, const float *v) {
            ((float4 *)d)[0] = make_float4(v[0], v[1], v[2], v[3]);
            ((float4 *)d)[1] = make_float4(v[4], v[5], v[6], v[7]);
        };
        if constexpr (F == FMT_F32) {
            put(p, hr);
            put(p + pstride, hi);
        } else {
            float lr[8], li[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                lr[q] = tf32_round(re[q] - hr[q]);
                li[q] = tf32_round(im[q] - hi[q]);
            }
            put(p, hr);
            put(p + pstride, lr);
            put(p + 2 * pstride, hi);
            put(p + 3 * pstride, li);
        }
    } else {
        using H = H16<F>;
        typename H::T *p = (typename H::T *)base + idx;
        __align__(16) typename H::T rh[8], ih[8], rl[8], il[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            rh[q] = H::hi(re[q]);
            ih[q] = H::hi(im[q]);
            rl[q] = H::from(re[q] - H::to(rh[q]));
            il[q] = H::from(im[q] - H::to(ih[q]));
        }
        if constexpr (F == FMT_BF16X2) {
            *(uint4 *)p = *(const uint4 *)rh;
            *(uint4 *)(p + pstride) = *(const uint4 *)ih;
        } else {
            *(uint4 *)p = *(const uint4 *)rh;
            *(uint4 *)(p + pstride) = *(const uint4 *)rl;
            *(uint4 *)(p + 2 * pstride) = *(const uint4 *)ih;
            *(uint4 *)(p + 3 * pstride) = *(const uint4 *)il;
        }
    }
}

// Stochastic splitting (BF16x3 form).  hi = SR(x) and lo = SR(x - hi), where SR
// rounds to bf16 up or down in magnitude with probability proportional to the
// distance (add random bits below the kept bits of the fp32 pattern, then
// truncate), so E[hi + lo] = x up to the randomness' granularity and the errors
// of different elements are independent and zero-mean: the products that a
// three-product split drops, and the rounding of the kept ones, then add up like
// sqrt(K) instead of K in a coherent sum.  A split takes 8 random bits per
// rounding: the bias left by that granularity is at most 2^-8 ulp, which puts the
// coherent part of the dropped lo*lo products near 2^-30 and that of lo's own
// rounding near 2^-23 of a sum's size, so one 32-bit hash serves both parts of
// both components of a complex element.  The bits come from a counter-based hash
// of the element's index and a per-operand seed (the 32-bit finaliser of
// MurmurHash3), so results are reproducible.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
// Two stochastic roundings to bf16 in one conversion (cvt.rs, sm_100 family): the upper half
// of the result is `a` with bits 31:16 of `rb` added below its kept bits (to the magnitude
// bits of the fp32 pattern) and truncated, the lower half `b` with bits 15:0.
__device__ __forceinline__ uint32_t cvt_bf16x2_sr(float a, float b, uint32_t rb) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rb));
    return d;
}
// 32 random bits for element `gidx` of the operand with seed `seed` (one finaliser
// round; the index's high word, zero for operands below 2^32 elements, is folded in
// by a multiply)
__device__ __forceinline__ uint32_t sr_word(uint64_t gidx, uint32_t seed) {
    const uint32_t k = (uint32_t)gidx ^ seed ^ ((uint32_t)(gidx >> 32) * 0x9e3779b9u);
    return fmix32(k);
}
// Split of one complex element, re + i im = (re_hi + re_lo) + i (im_hi + im_lo), with 8 random
// bits of r per rounding: bits 0-7 round re_hi, 8-15 re_lo, 16-23 im_hi, 24-31 im_lo (each
// placed at the top of its 16-bit addend).  Returns the packed pairs hi = (re_hi | im_hi << 16)
// and lo = (re_lo | im_lo << 16); x - hi is exact in fp32.
__device__ __forceinline__ void split_sr_cplx(float re, float im, uint32_t r, uint32_t &hi, uint32_t &lo) {
    hi = cvt_bf16x2_sr(im, re, ((r & 0x00ff0000u) << 8) | ((r & 0x000000ffu) << 8));
    const float re_h = __uint_as_float(hi << 16), im_h = __uint_as_float(hi & 0xffff0000u);
    lo = cvt_bf16x2_sr(im - im_h, re - re_h, r & 0xff00ff00u);
}
// Packs the low (re) halves and the high (im) halves of two split pairs: (x0.re | x1.re << 16)
// and (x0.im | x1.im << 16).
__device__ __forceinline__ uint32_t pack_re(uint32_t x0, uint32_t x1) { return __byte_perm(x0, x1, 0x5410); }
__device__ __forceinline__ uint32_t pack_im(uint32_t x0, uint32_t x1) { return __byte_perm(x0, x1, 0x7632); }

// store_cplx for the BF16X4 layout with stochastic splitting (element index gidx)
__device__ __forceinline__ void store_cplx_sr(void *base, size_t pstride, size_t idx, float re, float im, uint64_t gidx,
                                              uint32_t seed) {
    unsigned short *p = (unsigned short *)base;
    uint32_t hi, lo;
    split_sr_cplx(re, im, sr_word(gidx, seed), hi, lo);
    p[idx] = (unsigned short)hi;
    p[pstride + idx] = (unsigned short)lo;
    p[2 * pstride + idx] = (unsigned short)(hi >> 16);
    p[3 * pstride + idx] = (unsigned short)(lo >> 16);
}

// Eight split elements (element q has index gidx + q) as four packed 16-byte rows: re_hi,
// re_lo, im_hi, im_lo.
__device__ __forceinline__ void split8_sr(const float (&re)[8], const float (&im)[8], uint64_t gidx, uint32_t seed,
                                          uint4 &rh, uint4 &rl, uint4 &ih, uint4 &il) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) split_sr_cplx(re[q], im[q], sr_word(gidx + q, seed), hi[q], lo[q]);
    rh = make_uint4(pack_re(hi[0], hi[1]), pack_re(hi[2], hi[3]), pack_re(hi[4], hi[5]), pack_re(hi[6], hi[7]));
    rl = make_uint4(pack_re(lo[0], lo[1]), pack_re(lo[2], lo[3]), pack_re(lo[4], lo[5]), pack_re(lo[6], lo[7]));
    ih = make_uint4(pack_im(hi[0], hi[1]), pack_im(hi[2], hi[3]), pack_im(hi[4], hi[5]), pack_im(hi[6], hi[7]));
    il = make_uint4(pack_im(lo[0], lo[1]), pack_im(lo[2], lo[3]), pack_im(lo[4], lo[5]), pack_im(lo[6], lo[7]));
}

// store_cplx8 for the BF16X4 layout with stochastic splitting; element q has index gidx + q
__device__ __forceinline__ void store_cplx8_sr(void *base, size_t pstride, size_t idx, const float (&re)[8],
                                               const float (&im)[8], uint64_t gidx, uint32_t seed) {
    __nv_bfloat16 *p = (__nv_bfloat16 *)base + idx;
    uint4 rh, rl, ih, il;
    split8_sr(re, im, gidx, seed, rh, rl, ih, il);
    *(uint4 *)p = rh;
    *(uint4 *)(p + pstride) = rl;
    *(uint4 *)(p + 2 * pstride) = ih;
    *(uint4 *)(p + 3 * pstride) = il;
}

// Read back the value an operand represents (hi + lo).
template <int F>
__device__ __forceinline__ float2 load_cplx(const void *base, size_t pstride, size_t idx) {
    if constexpr (F == FMT_F32) {
        const float *p = (const float *)base;
        return make_float2(p[idx], p[pstride + idx]);
    } else if constexpr (F == FMT_BF16X4 || F == FMT_F16X4) {
        using H = H16<F>;
        const typename H::T *p = (const typename H::T *)base;
        return make_float2(H::to(p[idx]) + H::to(p[pstride + idx]), H::to(p[2 * pstride + idx]) + H::to(p[3 * pstride + idx]));
    } else if constexpr (F == FMT_BF16X2) {
        const __nv_bfloat16 *p = (const __nv_bfloat16 *)base;
        return make_float2(__bfloat162float(p[idx]), __bfloat162float(p[pstride + idx]));
    } else {
        const float *p = (const float *)base;
        return make_float2(p[idx] + p[pstride + idx], p[2 * pstride + idx] + p[3 * pstride + idx]);
    }
}

#define DLX_FMT_DISPATCH(fmt, F, ...)                                   \
    switch (fmt) {                                                      \
        case FMT_F32: { constexpr int F = FMT_F32; __VA_ARGS__; } break;     \
        case FMT_BF16X4: { constexpr int F = FMT_BF16X4; __VA_ARGS__; } break; \
        case FMT_BF16X2: { constexpr int F = FMT_BF16X2; __VA_ARGS__; } break; \
        case FMT_F16X4: { constexpr int F = FMT_F16X4; __VA_ARGS__; } break;   \
        default: { constexpr int F = FMT_TF32X4; __VA_ARGS__; } break;         \
    }

// Programmatic dependent launch.  The kernels of one evaluation run back to back
// on one stream, each launched with programmatic stream serialization.  No kernel
// signals early (griddepcontrol.launch_dependents): a CTA that exits counts as
// having signalled, so the next grid is launched as the last CTAs of the previous
// one exit, and its launch overlaps that tail.  Each kernel waits for the previous
// grid to finish and its writes to be visible (pdl_wait) before it touches global
// memory.  An early signal at kernel start was measured to cost more than it saved:
// the dependent grid's CTAs took the SMs freed by a multi-wave grid before its
// later waves ran (calibration workload 7.53 against 7.14 ms per back-to-back
// evaluation, binary star 0.766 against 0.699 ms).  Without a programmatic
// dependency pdl_wait is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// 2^-ceil(log2 x) for finite x > 0 (so that x times it lies in (1/2, 1]), else 1:
// the power-of-two operand scales of the FP16 form.
__host__ __device__ inline float inv_pow2_ceil(float x) {
    if (!(x > 0.f) || !(x < 3.0e38f)) return 1.f;
    int e = 0;
    const float m = frexpf(x, &e);  // x = m 2^e, m in [1/2, 1)
    return ldexpf(1.f, m == 0.5f ? 1 - e : -e);
}

// One operand tensor (plane-major [batch][planes][rows][ld]) and its TMA map.
struct Operand {
    void *ptr = nullptr;
    int batch = 0, rows = 0, ld = 0;  // ld = padded contraction length
    int planes = 0;                   // planes of this operand (the plan's form, or 2 for hi-only ones)
    size_t bytes = 0;
    CUtensorMap tmap;                 // valid when the plan uses a tensor-core form
    CUtensorMap tmap_hi;              // split operands of the BF16x3sa form: the hi planes (re_hi, im_hi) only
};

// Parameters of R independent same-shape models ("slots"): array k of slot r
// starts at p[k] + r * s[k] (s[k] = 0 shares one array between slots).
enum { PT = 0, POPDF, PBASIS, PCOEFF, POPDPIX, PW, PFLUX, PPOS, PDITHER, PFLAT, NPARAM };
struct DevParams {
    const float *p[NPARAM];
    size_t s[NPARAM];
};
enum { GZERN = 0, GPIX, GFLAT, GFLUX, GPOS, NGRAD };
struct DevGrads {
    float *p[NGRAD];
    size_t s[NGRAD];
};

__device__ __forceinline__ const float *slot_ptr(const DevParams &P, int k, int r) {
    return P.p[k] ? P.p[k] + (size_t)r * P.s[k] : nullptr;
}

}  // namespace dlx

// A plan holds the MFT matrices of one shape and wavelength set and the
// workspaces for up to R_max slots.  PSF index: bg = r * B + l * nse + s * ne + e.
struct dlx_plan {
    dlx_mft_desc desc;
    std::vector<double> lambdas;
    int device = 0, sm_count = 0, cc_major = 0, cc_minor = 0;
    int R_max = 1;
    int ni, nd, os, no, nl, ns, ne, nz, B, nse, ldi, ldo;  // nd, ne, no: the MFT's detector
    // the images: ndi x ndi pixels, nei of them.  Equal to nd, ne unless the dithers are integer
    // pixels (desc.dither_px): then the MFT runs once per source on nd = ndi + 2 max|dither| with
    // ne = 1, and image e is the window of it at crop[e] (device int2 (x, y) offsets, pixels)
    int ndi, nei;
    int *crop = nullptr;
    std::vector<int32_t> dither_px;  // host copy of desc.dither_px ([nei][2]) or empty
    int prec, fmt, planes, esz;
    double dx, du;   // du: the transform's angle step, (pixscale / os) f / z in the Fresnel regime
    double chirp = 0.0;  // Fresnel regime: (1/z - 1/f) / 2, the pupil's quadratic phase is 2 pi chirp |x|^2 / lambda
    int G = 1;       // partial-intensity planes of the intensity contraction
    // tensor-core forms: the intensity contraction's work split for R active slots
    // (s2[R-1]); offsets and pieces live in s2_table (see s2_schedule.h)
    struct S2Split {
        long off = 0, pcs = 0;  // int offsets of the CTA offsets and of the pieces
        int nct = 0, npieces = 0;
        long fold = 0;          // int2 offset of this split's fold list in s2_fold
        int nfold = 0;          // segments written in more than one plane
        long used = 0;          // byte offset of this split's plane counts in s2_used
    };
    // Tensor-core forms: the split clears none of the planes a segment leaves unwritten.
    // Up to 8 sources the one-pass binning and the PSF output read each segment's planes as
    // counted in s2_used ([rse][tile] per split); beyond 8, where the binning reads the
    // intensity twice, k_plane_fold first adds the (segment, planes written) pairs of
    // s2_fold into plane 0 and the readers take plane 0 alone.
    int *s2_fold = nullptr;
    uint8_t *s2_used = nullptr;
    std::vector<S2Split> s2;
    int *s2_table = nullptr;
    int chunk = 1;   // PSFs per adjoint pass
    int gsplit = 1;  // K splits of the adjoint 1^T contraction: gphi holds [R*B][gsplit][ni*ni]
    dlx::Operand amat, amatH, P, T1t, GEt, GT1;
    // Mirror-paired forward (the FP16 split form, see pair_layout below): amat holds [Re A | Im A]
    // over the first half of the pupil axis in two planes (hi, lo), Pp the phasor's mirror sums
    // and differences along both pupil axes, and T1t the first-stage product in the same paired
    // layout along its pupil axis; P keeps the plain phasor for the adjoint 1^T epilogue.
    bool paired = false;
    int hn = 0, hp = 0;        // pair indices ceil(Ni/2), and that count rounded up to 16
    int ldk = 0;               // row length of the paired operands: operand_ld(2 hp)
    dlx::Operand Pp;
    // Mirror-paired adjoint (paired plans that keep stage 2's field): the same pairing along the
    // output axes.  amatH holds [Re A^H | Im A^H] over the first half of the output axis (two
    // planes), GEt the adjoint field paired along kx (rows) and ky (columns), GT1 the adjoint 2^T
    // product paired along kx (columns), as Pp and T1t are paired on the pupil axes.
    bool padj = false;
    int hno = 0, hpo = 0, ldko = 0;  // ceil(No/2), rounded up to 16, operand_ld(2 hpo)
    double *lam_d = nullptr;   // [nl]
    float *wnorm = nullptr;    // [R][nl] weights / sum(weights)
    float *pscale = nullptr;   // [R][2] 1/sqrt(sum T^2), FP16 phasor scale pi_r
    float *tpart = nullptr;    // [R][kNormParts] block maxima of |T|
    float *ascale = nullptr;   // [nl] FP16 MFT-matrix scales alpha_l (FP16 form)
    unsigned int *qmax = nullptr;  // [R][nse] FP16 form: max_q |GI| sqrt(I_se(q)) (float bits)
    unsigned int *gmax = nullptr;  // [R*B] FP16 form: max |GEt'| per PSF (float bits)
    float *invlam = nullptr;   // [nl] 1/lambda (FP32)
    float2 *tilt = nullptr;    // [R*B][2][ni]
    float *opd = nullptr;      // [R][ni*ni]
    float *Is = nullptr;       // [G][R*nse][no][no] per-source intensity partials
    float *Ef = nullptr;       // [R*B][re, im][no][ldo] fp32 fields kept by stage 2 for the adjoint, or NULL
    float *GIt = nullptr;      // [R][ne][nd][nd] GI transposed (x rows, y columns), with Ef
    float *GI = nullptr;       // [R][ne][nd*nd] FF * dL/dm on the MFT's detector
    float *GIimg = nullptr;    // integer dithers: [R][nei][ndi*ndi] the images' FF * dL/dm
    float *Swin = nullptr;     // integer dithers: [R][nd*nd] sum_s F_s B_s on the big detector
    float *model_tmp = nullptr;// [R][nei][ndi*ndi]
    float *gphi = nullptr;     // [R*B][ni*ni] (2 pi / lambda) dL/dphase
    float2 *gopd = nullptr;    // [R][ni*ni] g_OPD as a compensated (hi, lo) FP32 pair
    double *red = nullptr;     // [R][red_blocks][1 + kMaxSrc] reduction partials (up to 8 sources)
    int red_blocks = 0;
    // more than 8 sources: two-pass binning (k_bin_model, k_flux_grad) and its partials
    int bin_a_blocks = 1, bin_b_blocks = 1;
    double *red_a = nullptr;   // [R][bin_a_blocks] loss partials
    double *red_b = nullptr;   // [R][kMaxSrc][bin_b_blocks] flux-gradient partials
    unsigned int *fcount = nullptr;  // [R][kMaxSrc] finished flux-gradient blocks (reset by the last)
    double *pos_part = nullptr;// CUDA-core form: [R*B][gsplit][2] position-moment partials
    float2 *zpart = nullptr;   // [R][n_zern][ceil(Ni^2 / 64)] Zernike-gradient partials (compensated pairs)
    unsigned int *bcount = nullptr;  // [R] blocks of the binning pass done (reset by the last one)
    float *mom = nullptr;      // tensor-core forms: [R*B][gsplit][tiles][8 warps][2] position moments
    uint32_t sr = 0;           // BF16x3 forms: stochastic splitting of the forward operands (seed base), else 0
    bool adj1 = false;         // BF16x3sa: the adjoint contracts the stochastic hi parts only (2-plane bf16)
    // set by eval_loss_grad for one evaluation: stage 2 also writes every PSF's field E (Ef) and
    // the adjoint forms its field operand from it instead of recomputing it
    bool keep_field = false;
    float prf_inv = 0.f;       // 1 / sigma^2 of the chi^2 prior on the flat field, 0 = none
    // forward-mode derivative (dlx_model_jvp): while tan_map is set, the phasors of the sources
    // in tan_mask are multiplied by (1 + i tan_coef (2 pi / lambda) tan_map[n])
    const float *tan_map = nullptr;
    float tan_coef = 0.f;
    uint32_t tan_mask = 0;
    // vector-Jacobian product (dlx_model_vjp): while set, the adjoint weights dL/dm are this
    // cotangent [n_exp][Nd][Nd] instead of 1 - d/m
    const float *cot = nullptr;
    float2 *npart = nullptr;   // [R][kNormParts] block partials of sum T^2 (compensated pairs)
    unsigned int *ncount = nullptr;  // [R] blocks of the prologue pass done (reset by the last one)
    int32_t *err = nullptr;    // device error flag
    unsigned long long *clamped = nullptr;
    size_t workspace = 0;
    std::vector<void *> allocs;
    // per-kernel-class timing (events on the launching stream) and launch counts
    struct TimedRec {
        int cls;
        cudaEvent_t a, b;
    };
    uint32_t timing = 0;  // bit c: time kernel class c
    std::vector<TimedRec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_next = 0;
    int64_t launches[16] = {};
    int64_t events[16] = {};
    // checked mode, level 2: the first kernel class that failed in the current call
    int check_rc = 0;
    std::string check_msg;
    int inject = 0;  // test hook (dlx_plan_inject_fault): 1 = withhold an operand copy in the next contraction
};

namespace dlx {

constexpr int kMaxSrc = 32;  // sources per plan
// Row length of the operand planes: a multiple of 64 elements, so that every 64-byte row chunk a
// TMA box reads starts on a 64-byte boundary (with 1064-element rows, 2128-byte pitch, the chunks of
// odd rows straddled 32-byte sectors and the L2 served the adjoint contractions at 1.3 sectors
// per request instead of 2).  The padding columns are zero.
inline int operand_ld(int n) { return (n + 63) / 64 * 64; }
constexpr int kMinBf16Pupil = 32;  // smallest pupil (samples per side) the BF16 split forms run at

// Mirror pairing of the forward contractions (the two-sided MFT of Sec. 3 on the centred grids
// x_n = (n - (Ni-1)/2) dx, u_k = (k - (No-1)/2) du).  Since x_{Ni-1-n} = -x_n, the matrix has
// A[k][Ni-1-n] = conj(A[k][n]), so for any row v along the pupil axis, with j < hn = ceil(Ni/2),
// m = Ni-1-j, S_j = v_j + v_m, D_j = v_j - v_m (S = v_j, D = 0 for the middle of an odd axis,
// where A is real):
//   sum_n A[k][n] v_n = sum_j a[k][j] S_j + i b[k][j] D_j,   a = Re A, b = Im A,
// so  Re = sum_j a S_re - b D_im  and  Im = sum_j a S_im + b D_re.  Each is a real contraction of
// the matrix row [a | b] (length 2 hp, each half padded with zeros to hp = hn rounded up to 16)
// with a varying row [S_re | D_im] or [S_im | D_re], the second half of the first one subtracted:
// six tensor-core products per 16-wide step of a (hi, lo) split instead of twelve for the complex
// product, on the same operand bytes.  The sums and differences are rounded to the split in place
// of the samples, at up to twice their modulus, which raises the split's representation error by
// a factor near 1.4: the FP16 split (about 2^-20) absorbs that, the BF16 split (2^-17, BF16x3
// already near 1e-5 of the PSF peak) does not, so only the FP16 split form is paired.  The
// paired layouts:
//   amat (forward matrix)  [nl][hi, lo][No][ldk]:  row k = [a[k][0..hn) 0.. | b[k][0..hn) 0..];
//   T1t (stage-1 product)  [B][V1 hi, V1 lo, V2 hi, V2 lo][No][ldk], for stage 2 (the pupil-y
//      axis): column R hp + j (R = 0 for S, 1 for D) of row kx holds T1_R[kx][j], the first-stage
//      product of the y-paired phasor rows, as V1 = Re, V2 = Im for S and V1 = Im, V2 = Re for D;
//   Pp (phasor)            [B][V1 hi, V1 lo, V2 hi, V2 lo][2 hp][ldk]: row Ry hp + jy, column
//      Rx hp + jx holds the phasor paired along y (rows) and along x (columns), placed as in T1t
//      by Rx.
// Stage 1 applied to the y-paired rows of Pp gives T1_S and T1_D directly (the contraction is
// linear), so no pass forms the pairs of its output.
inline int pair_half(int n) { return ((n + 1) / 2 + 15) / 16 * 16; }
constexpr int kNormParts = 1024;  // maximum blocks of the OPD / pupil-power pass

enum KClass { KC_MATRICES = 0, KC_PROLOGUE, KC_STAGE1, KC_STAGE2, KC_BIN, KC_LOSS, KC_ADJ_FIELD, KC_ADJ2, KC_ADJ1,
              KC_GRAD, KC_ADAM, KC_FIELD_SCALE, KC_N };

// Checked mode (dlx_set_checks): the process-wide level, and the level-2 check after a
// kernel class (synchronises the stream unless it is being captured; records the first
// failure in p->check_rc / p->check_msg).
int check_level();
void class_check(dlx_plan *p, int cls, cudaStream_t st);
const char *class_name(int cls);
// Level-1 checks: one array (NULL passes when `optional`), the arrays of dlx_params and of
// dlx_grads for plan p, and the bytes of one [nei][ndi][ndi] image set of 4-byte elements.
int check_buffer(const void *ptr, size_t bytes, size_t align, int device, const char *name, bool optional);
int check_params(const dlx_plan *p, const dlx_params *q);
int check_grads(const dlx_plan *p, const dlx_grads *g, const char *what);
size_t image_bytes(const dlx_plan *p);
// A call's status after its launches: a level-2 failure recorded on the plan replaces OK.
int checked_status(dlx_plan *p, int rc);

// Scope around one class of launches on stream st: counts the `n` kernels it
// launches and, when the plan's timing is on, records events around them.
struct KScope {
    dlx_plan *p;
    int cls, n;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    KScope(dlx_plan *p, int cls, int n, cudaStream_t st);
    ~KScope();
};

// the tensor-core split's planes are folded into plane 0 after stage 2 (more than 8 sources,
// or integer-dither windows)
inline bool folds_planes(const dlx_plan *p) { return p->prec != DLX_FP32_SIMT && (p->ns > 8 || p->crop); }
// row blocks of k_win_flux: about 16 blocks of 128 threads per SM over columns x rows x sources
inline int win_flux_rows(const dlx_plan *p, int R) {
    const int cx = (p->nd + 127) / 128;
    return std::max(1, std::min(p->nd, p->sm_count * 16 / (cx * p->ns * R)));
}
// partial-intensity planes a reader adds (at most; see plane_counts)
inline int planes_to_read(const dlx_plan *p) { return folds_planes(p) ? 1 : p->G; }
// the plane-count table for R active slots where the readers need it, else NULL
inline const uint8_t *plane_counts(const dlx_plan *p, int R) {
    return (!folds_planes(p) && p->s2_used && R >= 1 && R <= (int)p->s2.size()) ? p->s2_used + p->s2[R - 1].used
                                                                                  : nullptr;
}

// Fresnel regime of a descriptor (focal_length_m > 0, detector at z = f + focal_shift_m): the
// factor on the transform's angle step (f / z) and the pupil chirp coefficient (1/z - 1/f) / 2;
// (1, 0) in the Fraunhofer regime.
inline void fresnel_terms(const dlx_mft_desc *d, double *du_scale, double *chirp) {
    *du_scale = 1.0;
    *chirp = 0.0;
    if (d->focal_length_m > 0) {
        const double f = d->focal_length_m, z = f + d->focal_shift_m;
        *du_scale = f / z;
        *chirp = 0.5 * (1.0 / z - 1.0 / f);
    }
}

// ---- plan construction (dlx_api.cu)
// Validates a descriptor (sizes, ranges, wavelengths, precision, Fresnel terms, dithers):
// DLX_OK, or the status with dlx_last_error set; *delta_out = max |dither_px| (may be NULL).
int check_desc(const dlx_mft_desc *d, int *delta_out);
int make_plan(const dlx_mft_desc *d, int device, int R_max, dlx_plan **out);
void free_plan(dlx_plan *p);

// ---- launchers (k_elem.cu); R = number of active slots (<= R_max)
cudaError_t launch_mft_matrices(dlx_plan *p, cudaStream_t st);
cudaError_t launch_prologue(dlx_plan *p, const DevParams &prm, int R, cudaStream_t st);  // OPD, norm, tilt, phasor
// binning + flat field (+ Poisson NLL and its partials when data != NULL)
// with data, the last block also writes loss[r] (may be NULL) and dL/dF_s
cudaError_t launch_bin_nll(dlx_plan *p, const DevParams &prm, int R, const int32_t *data, size_t data_stride,
                           float *model, size_t model_stride, const DevGrads *g, double *loss, cudaStream_t st);
cudaError_t launch_psf_out(dlx_plan *p, const DevParams &prm, float *psf, cudaStream_t st);
cudaError_t launch_grad_reduce(dlx_plan *p, const DevParams &prm, int R, const DevGrads *g, cudaStream_t st);
cudaError_t launch_adam(float *theta, const float *grad, float *m, float *v, size_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t st);
// F = J diag(w) J^T (dlx_fisher_gram); work holds DLX_GRAM_BLOCKS x n(n+1)/2 doubles
cudaError_t launch_fisher_gram(const float *J, int n, size_t npix, const float *model, const int32_t *data, double *F,
                               double *work, cudaStream_t st);
// cot = 1 - d / max(m, 1e-30) elementwise (dlx_nll_cotangent)
cudaError_t launch_nll_cotangent(const float *m, const int32_t *d, size_t n, float *cot, cudaStream_t st);
// adds the stage-2 split's extra planes into plane 0 (tensor-core forms; no-op otherwise)
cudaError_t launch_plane_fold(dlx_plan *p, int R, cudaStream_t st);
// Whether an evaluation of R slots keeps the fields stage 2 forms for the adjoint: plans of the
// split forms (BF16x3, BF16x4, FP16x3, TF32x3; not BF16x3sa) and of the FP32 CUDA-core form whose
// adjoint operand holds every PSF at once allocate Ef.
inline bool keeps_field(const dlx_plan *p, int R) { return p->Ef != nullptr && p->chunk >= R * p->B; }
// Whether a plan of this form, pupil size, PSF count and adjoint chunk allocates Ef (the FP16
// form's mirror-paired adjoint needs the kept field: its scaling pass writes the paired operand).
inline bool field_kept(int fmt, bool adj1, int ni, int chunk, int Bt) {
    (void)ni;
    return (fmt == FMT_BF16X4 || fmt == FMT_F16X4 || fmt == FMT_TF32X4 || fmt == FMT_F32) && !adj1 && chunk >= Bt;
}
// The adjoint field from the kept fields: GEt[z] = split(2 w F GI o Ef[b0 + z]) (z < nb).
cudaError_t launch_field_scale(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st);
// a = (a - b) * c elementwise (the central difference of dlx_model_jvp)
cudaError_t launch_scaled_diff(float *a, const float *b, size_t n, float c, cudaStream_t st);
// Adam over R packed slots of n parameters each; group k of a slot is
// [off[k], off[k+1]) with learning rate lr[r][k]; step[r] is 1-based.
cudaError_t launch_adam_slots(float *theta, const float *grad, float *m, float *v, size_t n, int R, const int *off,
                              const float *lr, const int *step, float b1, float b2, float eps, cudaStream_t st);

// ---- contractions (k_gemm_simt.cu / k_gemm_tc.cu) over global PSF indices
// stage 1:  T1t[bg] = A(l) . P[bg]^T                   (rows kx, cols ny)
// stage 2:  Is[g][r nse + se] = sum_{l in g} w_l |A(l) . T1t[bg]^T|^2
// adjoint:  GEt[z] = 2 w_l F_s GI o (T1t[bg] . A(l)^T),  GT1[z] = AH(l) . GEt[z]^T,
//           gphi[bg] = (2 pi/lambda) Im((GT1[z] . AH(l)^T) conj P[bg]),   z = bg - b0
cudaError_t simt_forward(dlx_plan *p, int R, cudaStream_t st);
cudaError_t simt_adjoint_chunk(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st);
cudaError_t tc_forward(dlx_plan *p, int R, cudaStream_t st);
cudaError_t tc_adjoint_chunk(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st);
int tc_supported(const dlx_plan *p, std::string *why);
int tc_make_maps(dlx_plan *p, std::string *why);

// ---- whole evaluations (dlx_api.cu), asynchronous on st
int eval_forward(dlx_plan *p, const DevParams &prm, int R, cudaStream_t st);
int eval_loss_grad(dlx_plan *p, const DevParams &prm, int R, const int32_t *data, size_t data_stride, double *loss,
                   const DevGrads *g, float *model, size_t model_stride, cudaStream_t st);

}  // namespace dlx

// error reporting (dlx_api.cu)
void dlx_set_error(const std::string &msg);
