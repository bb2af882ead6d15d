// Tensor-core form of the four MFT contractions (Sec. 3, two-sided MFT) on
// sm_103a: TMA -> shared memory -> tcgen05.mma -> tensor memory -> epilogue.
//
// Every contraction is C[m][n] = sum_k A[m][k] B[n][k] over complex operands
// held as bf16 (or tf32) planes, both K-major.  One CTA (320 threads) owns a
// 128 x 128 complex output tile per job and runs persistently over jobs:
//   warp 8  : TMA producer (one lane) -- 4-D tensor maps {k, row, plane, batch},
//             64-byte swizzled boxes of every plane of A and B per stage;
//   warp 9  : MMA issuer (one lane) and tensor-memory owner -- per 16-wide k
//             step it issues the complex product as real products into FP32
//             accumulators in tensor memory (the subtraction in Re(AB) is the
//             instruction descriptor's negate-A bit);
//   warps 0-7: epilogue -- tcgen05.ld of a 32-lane quarter and a 64-column
//             half of the accumulators, 16 columns at a time, then the
//             contraction's fused epilogue (operand split store, spectral
//             |E|^2 accumulation, dL/dE scaling, or the phase-gradient product
//             with conj(P)).
// The kernel is specialised per contraction kind, arithmetic form and
// accumulation mode, so each instance carries only its own epilogue.
// Every mbarrier wait is bounded (globaltimer, 1 s): on expiry the CTA raises
// a shared abort flag and the plan's device error flag, waits (bounded) for
// its own copies and MMAs in flight, frees its tensor memory and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "dlx_common.cuh"

namespace dlx {
namespace {

constexpr int BM = 128, BN = 128, NTHREADS = 320, EPI_WARPS = 8, PRODUCER_WARP = 8, MMA_WARP = 9;
constexpr int PLANE_BYTES = 128 * 64;  // one 128-row x 64-byte swizzled box
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;
constexpr uint32_t TMEM_COLS = 512;
constexpr int CW = 16;  // epilogue columns per tensor-memory load

enum Kind { KS1 = 0, KS2 = 1, KGE = 2, KGT1 = 3, KGP = 4 };

// Accumulation modes.  FAST: two accumulators (Er, Ei), double-buffered, three
// split products.  SPLIT3 / SPLIT4: the hi*hi products and the small correction
// products go to separate accumulators (Er_hh, Ei_hh, Er_c, Ei_c; one buffer),
// so the accumulator that carries the large values takes two instructions per
// 16-wide k step instead of six -- the tensor core's FP32 accumulation loses a
// fraction of an ulp towards zero per instruction, and at a PSF peak those
// losses add up coherently.  SPLIT4 also adds the lo*lo product, whose omission
// biases coherent sums of conjugate pairs upwards by about 2^-16.
enum AccMode { FAST = 0, SPLIT3 = 1, SPLIT4 = 2 };

template <int F>
struct Cfg {
    static constexpr int PL = fmt_planes(F);
    static constexpr int ES = fmt_esize(F);
    static constexpr int KB = 64 / ES;  // k elements per stage (64 bytes per row)
    static constexpr int STAGE_BYTES = 2 * PL * PLANE_BYTES;
    static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
    static constexpr int KSTEP = (F == FMT_TF32X4) ? 8 : 16;  // k per MMA instruction (32 bytes)
    static constexpr int NKSTEP = KB / KSTEP;
    static constexpr uint32_t AB_FMT = (F == FMT_TF32X4) ? 2u : (F == FMT_F16X4) ? 0u : 1u;  // TF32 : F16 : BF16
    // 16-bit forms stage the operand tiles they write in one swizzled TMA box
    // (128 rows x 64 bytes x all planes) and store them with bulk tensor copies
    static constexpr bool TMA_STORE = (F == FMT_BF16X4 || F == FMT_BF16X2 || F == FMT_F16X4);
    static constexpr int STG_BYTES = TMA_STORE ? PL * PLANE_BYTES : 0;
    static constexpr int SMEM = STAGES * STAGE_BYTES + STG_BYTES + 1024 + 256;
};

// Shared-memory stages of one launch.  Mirror-paired contractions (PR, the FP16 split form;
// pair_layout in dlx_common.cuh) read a two-plane matrix operand (hi, lo of [Re A | Im A] or of
// [Re A^H | Im A^H]): the A operand of stage 1, stage 2 and the adjoint 2^T, the B operand of the
// recomputed field and the adjoint 1^T.
template <int F, int PR, int KIND>
struct Geo {
    static constexpr int PA = (PR && (KIND == KS1 || KIND == KS2 || KIND == KGT1)) ? 2 : Cfg<F>::PL;
    static constexpr int PB = (PR && (KIND == KGE || KIND == KGP)) ? 2 : Cfg<F>::PL;
    static constexpr int STAGE_BYTES = (PA + PB) * PLANE_BYTES;
    static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + Cfg<F>::STG_BYTES + 1024 + 256;
};

// Arguments of one launch.  Per-job operand coordinates come from decode().
struct TcArgs {
    int M, N, K;   // per-job contraction sizes (complex)
    int tm, tn;    // 128-tiles along M and N
    int units;
    int ksplit;    // K splits of the adjoint 1^T contraction (gphi planes per PSF)
    int KB;        // k elements per pipeline stage
    int nl, nse, B, ne, nd, os, ni, no, ldi, ldo, G, Rnse, b0;
    const float *wnorm;
    const float *GI;
    DevParams prm;
    float *Is;
    void *out;        // operand output base (KS1, KGE, KGT1)
    int out_ld;
    size_t out_ps;    // plane stride (elements)
    const void *P;    // phasor operand (KGP)
    const double *lam;
    float *gphi;
    float *mom;       // per-warp position moments (KGP)
    float dxf, cNf;   // pupil spacing and centre index (KGP)
    // FP16 form: operand scales (all powers of two) -- alpha_l, (1/sqrt(sum T^2), pi_r)
    // per slot, sigma1 of T1t, the adjoint-field bound maxima and per-PSF max |GEt'|
    const float *ascale, *pscale;
    float sig1;
    const unsigned int *qmax;
    unsigned int *gmax;
    const int *s2off; // stage 2: CTA c runs pieces s2pc[s2off[c] .. s2off[c+1])
    const int4 *s2pc; // stage 2 pieces (segment, l0, l1, plane | first plane to clear << 16)
    int grid;         // CTAs (0: min(units, SMs))
    uint32_t sr;      // BF16x3 forms: stochastic split (seed) of the operand this launch writes, else 0
    int p4;           // BF16x3sa adjoint 1^T: the phasor is a four-plane split
    int hp;           // mirror-paired contractions: the second half of K starts at hp
    int stall;        // test hook: CTA 0 withholds its first operand copy (its waits expire, bounded)
    int32_t *err;
};

struct Job {
    int a_batch, a_row, b_batch, b_row;
    int m0, n0;
    int b;       // global PSF index
    int z;       // chunk-local index
    int l, r, se;
    int kb0, kb1;  // k-block range of this job (split-K for the adjoint 1^T contraction)
    int split;
};

// Units of this CTA: stage 2 runs its pieces of the host-built split (see
// s2_schedule.h); every other contraction takes units blockIdx.x + k gridDim.x.
template <int KIND>
__device__ __forceinline__ void unit_range(const TcArgs &a, int &u0, int &u1, int &du) {
    if constexpr (KIND == KS2) {
        u0 = __ldg(a.s2off + blockIdx.x);
        u1 = __ldg(a.s2off + blockIdx.x + 1);
        du = 1;
    } else {
        u0 = blockIdx.x;
        u1 = a.units;
        du = gridDim.x;
    }
}

// Jobs of unit u (stage 2: the wavelengths of its piece `pc`).
template <int KIND>
__device__ __forceinline__ int decode_unit_jobs(const TcArgs &a, int u, int4 &pc) {
    if constexpr (KIND != KS2) {
        return 1;
    } else {
        pc = __ldg(a.s2pc + u);
        return pc.z - pc.y;
    }
}

template <int KIND>
__device__ __forceinline__ Job decode(const TcArgs &a, int u, int j, const int4 &pc) {
    Job J;
    const int tt = a.tm * a.tn;
    int tile = u % tt;
    J.split = 0;
    if constexpr (KIND == KS2) {
        // segment = (slot, source, exposure) x tile, tile fastest
        tile = pc.x % tt;
        const int rse = pc.x / tt;
        J.l = pc.y + j;
        J.r = rse / a.nse;
        J.se = rse % a.nse;
        J.b = J.r * a.B + J.l * a.nse + J.se;
        J.z = 0;
        J.a_batch = J.l;  // A(l) . T1t[b]^T
        J.b_batch = J.b;
    } else {
        int z = u / tt;
        if constexpr (KIND == KGP) {  // units are (z, tile, split) with the split fastest
            J.split = u % a.ksplit;
            const int rest = u / a.ksplit;
            tile = rest % tt;
            z = rest / tt;
        }
        J.z = z;
        J.b = (KIND == KS1) ? z : a.b0 + z;
        J.r = J.b / a.B;
        J.l = (J.b % a.B) / a.nse;
        J.se = (J.b % a.B) % a.nse;
        if constexpr (KIND == KS1) {  // A(l) . P[b]^T
            J.a_batch = J.l;
            J.b_batch = J.b;
        } else if constexpr (KIND == KGE) {  // T1t[b] . A(l)^T
            J.a_batch = J.b;
            J.b_batch = J.l;
        } else if constexpr (KIND == KGT1) {  // AH(l) . GEt[z]^T
            J.a_batch = J.l;
            J.b_batch = J.z;
        } else {  // GT1[z] . AH(l)^T
            J.a_batch = J.z;
            J.b_batch = J.l;
        }
    }
    J.m0 = (tile / a.tn) * BM;
    J.n0 = (tile % a.tn) * BN;
    J.a_row = J.m0;
    J.b_row = J.n0;
    const int nkb = (a.K + a.KB - 1) / a.KB;
    if constexpr (KIND == KGP) {
        J.kb0 = (int)((long)J.split * nkb / a.ksplit);
        J.kb1 = (int)((long)(J.split + 1) * nkb / a.ksplit);
    } else {
        J.kb0 = 0;
        J.kb1 = nkb;
    }
    return J;
}

// FP16 form: scale of the adjoint field operand of PSF b = (r, l, s, e).
// |G_E(q)| = 2 w_l F_s |GI(q)| |E(q)| <= 2 F_s sqrt(w_l) |GI(q)| sqrt(I_se(q)),
// since w_l |E_l(q)|^2 <= I_se(q) = sum_l w_l |E_l(q)|^2; gamma_b brings the bound
// to <= 1.
__device__ __forceinline__ float f16_gamma(const TcArgs &a, const Job &J) {
    const int s = J.se / a.ne;
    const float F = fabsf(slot_ptr(a.prm, PFLUX, J.r)[s]);
    const float w = fabsf(a.wnorm[(size_t)J.r * a.nl + J.l]);
    const float Q = __uint_as_float(a.qmax[(size_t)J.r * a.nse + J.se]);
    return inv_pow2_ceil(2.f * F * sqrtf(w) * Q);
}
// FP16 form: scale of the adjoint 2^T output GT1 of PSF b: |GT1 alpha gamma| <= No max |GEt'|.
__device__ __forceinline__ float f16_sigma2(const TcArgs &a, const Job &J) {
    return inv_pow2_ceil((float)a.no * __uint_as_float(a.gmax[J.b]));
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait.  Returns false when the limit expired (raising the abort flag and
// the device error) or when another role already aborted (unless `ignore_abort`).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int32_t *err, int code,
                          bool ignore_abort = false, uint64_t limit = WAIT_LIMIT_NS) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (!ignore_abort && *abort_flag) return false;
            if (gtimer() - t0 > limit) {
                *abort_flag = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// K-major operand in a 64-byte swizzled layout: rows of 64 bytes, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

template <int F>
__device__ __forceinline__ uint32_t idesc(bool negA) {
    return (1u << 4) | (Cfg<F>::AB_FMT << 7) | (Cfg<F>::AB_FMT << 10) | ((negA ? 1u : 0u) << 13) |
           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int F>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (F == FMT_TF32X4) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    }
}

// Bulk tensor store of a staged box, and the bulk-group bookkeeping around it.
__device__ __forceinline__ void tma_store4(const CUtensorMap *map, uint32_t src, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                     (uint64_t)map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Barrier of the 256 epilogue threads (warps 0-7).
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// The same barrier returning whether `v` holds for every epilogue thread.
__device__ __forceinline__ bool epi_all(bool v) {
    uint32_t out;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(out)
        : "r"((uint32_t)v)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive FP32 columns from tensor memory, waited on in the same asm.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ epilogue row I/O
// Store CW consecutive complex values of one row into a plane-major operand.
template <int F>
__device__ __forceinline__ void store_row(void *base, size_t ps, size_t off, const float (&re)[CW],
                                          const float (&im)[CW], int nvalid) {
    if (nvalid == CW) {
        if constexpr (F == FMT_BF16X4 || F == FMT_BF16X2 || F == FMT_F16X4) {
            using H = H16<F>;
            typename H::T *p = (typename H::T *)base + off;
#pragma unroll
            for (int q = 0; q < CW / 8; ++q) {
                __align__(16) typename H::T rh[8], ih[8], rl[8], il[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float x = re[8 * q + i], y = im[8 * q + i];
                    rh[i] = H::hi(x);
                    ih[i] = H::hi(y);
                    rl[i] = H::from(x - H::to(rh[i]));
                    il[i] = H::from(y - H::to(ih[i]));
                }
                if constexpr (F != FMT_BF16X2) {
                    *(uint4 *)(p + 8 * q) = *(uint4 *)rh;
                    *(uint4 *)(p + ps + 8 * q) = *(uint4 *)rl;
                    *(uint4 *)(p + 2 * ps + 8 * q) = *(uint4 *)ih;
                    *(uint4 *)(p + 3 * ps + 8 * q) = *(uint4 *)il;
                } else {
                    *(uint4 *)(p + 8 * q) = *(uint4 *)rh;
                    *(uint4 *)(p + ps + 8 * q) = *(uint4 *)ih;
                }
            }
        } else {
            float *p = (float *)base + off;
#pragma unroll
            for (int q = 0; q < CW / 4; ++q) {
                float4 h, l, hi, li;
                float *hp = &h.x, *lp = &l.x, *hip = &hi.x, *lip = &li.x;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float x = re[4 * q + i], y = im[4 * q + i];
                    hp[i] = split_hi8(x);
                    lp[i] = tf32_round(x - hp[i]);
                    hip[i] = split_hi8(y);
                    lip[i] = tf32_round(y - hip[i]);
                }
                *(float4 *)(p + 4 * q) = h;
                *(float4 *)(p + ps + 4 * q) = l;
                *(float4 *)(p + 2 * ps + 4 * q) = hi;
                *(float4 *)(p + 3 * ps + 4 * q) = li;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < CW; ++i)
            if (i < nvalid) store_cplx<F>(base, ps, off + i, re[i], im[i]);
    }
}

// Write 16 consecutive complex values of row r (columns 16h .. 16h+15 of a
// 32-column box) into the staged TMA box: planes of 128 rows x 64 bytes,
// 64-byte swizzle (16-byte granule g of row r sits at g ^ ((r >> 1) & 3)).
template <int F>
__device__ __forceinline__ void stage_row16(uint8_t *stg, int r, int h, const float (&re)[CW], const float (&im)[CW]) {
    using H = H16<F>;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        __align__(16) typename H::T rh[8], ih[8], rl[8], il[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float x = re[8 * q + i], y = im[8 * q + i];
            rh[i] = H::hi(x);
            ih[i] = H::hi(y);
            rl[i] = H::from(x - H::to(rh[i]));
            il[i] = H::from(y - H::to(ih[i]));
        }
        const int g = (2 * h + q) ^ ((r >> 1) & 3);
        uint8_t *p = stg + r * 64 + g * 16;
        if constexpr (F != FMT_BF16X2) {
            *(uint4 *)(p) = *(uint4 *)rh;
            *(uint4 *)(p + PLANE_BYTES) = *(uint4 *)rl;
            *(uint4 *)(p + 2 * PLANE_BYTES) = *(uint4 *)ih;
            *(uint4 *)(p + 3 * PLANE_BYTES) = *(uint4 *)il;
        } else {
            *(uint4 *)(p) = *(uint4 *)rh;
            *(uint4 *)(p + PLANE_BYTES) = *(uint4 *)ih;
        }
    }
}

// stage_row16 with the stochastic split of the BF16x3 form; element i of the
// row has global index gidx + i.
__device__ __forceinline__ void stage_row16_sr(uint8_t *stg, int r, int h, const float (&re)[CW], const float (&im)[CW],
                                               uint64_t gidx, uint32_t seed) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint4 rh, rl, ih, il;
        split8_sr(*(const float(*)[8])(re + 8 * q), *(const float(*)[8])(im + 8 * q), gidx + 8 * q, seed, rh, rl,
                  ih, il);
        const int g = (2 * h + q) ^ ((r >> 1) & 3);
        uint8_t *p = stg + r * 64 + g * 16;
        *(uint4 *)(p) = rh;
        *(uint4 *)(p + PLANE_BYTES) = rl;
        *(uint4 *)(p + 2 * PLANE_BYTES) = ih;
        *(uint4 *)(p + 3 * PLANE_BYTES) = il;
    }
}

// stage_row16 of a two-plane (re, im) bf16 operand with stochastic rounding (the
// BF16x3sa adjoint); element i of the row has global index gidx + i: 16 random bits
// per rounding, bits 15:0 of the element's word for re and 31:16 for im.
__device__ __forceinline__ void stage_row16_hi_sr(uint8_t *stg, int r, int h, const float (&re)[CW],
                                                  const float (&im)[CW], uint64_t gidx, uint32_t seed) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint32_t d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            d[i] = cvt_bf16x2_sr(im[8 * q + i], re[8 * q + i], sr_word(gidx + 8 * q + i, seed));
        const int g = (2 * h + q) ^ ((r >> 1) & 3);
        uint8_t *p = stg + r * 64 + g * 16;
        *(uint4 *)(p) = make_uint4(pack_re(d[0], d[1]), pack_re(d[2], d[3]), pack_re(d[4], d[5]), pack_re(d[6], d[7]));
        *(uint4 *)(p + PLANE_BYTES) =
            make_uint4(pack_im(d[0], d[1]), pack_im(d[2], d[3]), pack_im(d[4], d[5]), pack_im(d[6], d[7]));
    }
}

// Read CW consecutive complex values of one row of a plane-major operand
// (the value each represents: hi + lo).
template <int F>
__device__ __forceinline__ void load_row(const void *base, size_t ps, size_t off, float (&re)[CW], float (&im)[CW],
                                         int nvalid) {
    if (nvalid == CW) {
        if constexpr (F == FMT_BF16X4 || F == FMT_BF16X2 || F == FMT_F16X4) {
            using H = H16<F>;
            const typename H::T *p = (const typename H::T *)base + off;
#pragma unroll
            for (int q = 0; q < CW / 8; ++q) {
                __align__(16) typename H::T a[8], b[8], c[8], d[8];
                *(uint4 *)a = __ldg((const uint4 *)(p + 8 * q));
                if constexpr (F != FMT_BF16X2) {
                    *(uint4 *)b = __ldg((const uint4 *)(p + ps + 8 * q));
                    *(uint4 *)c = __ldg((const uint4 *)(p + 2 * ps + 8 * q));
                    *(uint4 *)d = __ldg((const uint4 *)(p + 3 * ps + 8 * q));
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        re[8 * q + i] = H::to(a[i]) + H::to(b[i]);
                        im[8 * q + i] = H::to(c[i]) + H::to(d[i]);
                    }
                } else {
                    *(uint4 *)c = __ldg((const uint4 *)(p + ps + 8 * q));
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        re[8 * q + i] = H::to(a[i]);
                        im[8 * q + i] = H::to(c[i]);
                    }
                }
            }
        } else {
            const float *p = (const float *)base + off;
#pragma unroll
            for (int q = 0; q < CW / 4; ++q) {
                const float4 h = __ldg((const float4 *)(p + 4 * q)), l = __ldg((const float4 *)(p + ps + 4 * q));
                const float4 hi = __ldg((const float4 *)(p + 2 * ps + 4 * q)),
                             li = __ldg((const float4 *)(p + 3 * ps + 4 * q));
                re[4 * q + 0] = h.x + l.x;
                re[4 * q + 1] = h.y + l.y;
                re[4 * q + 2] = h.z + l.z;
                re[4 * q + 3] = h.w + l.w;
                im[4 * q + 0] = hi.x + li.x;
                im[4 * q + 1] = hi.y + li.y;
                im[4 * q + 2] = hi.z + li.z;
                im[4 * q + 3] = hi.w + li.w;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < CW; ++i) {
            float2 v = make_float2(0.f, 0.f);
            if (i < nvalid) v = load_cplx<F>(base, ps, off + i);
            re[i] = v.x;
            im[i] = v.y;
        }
    }
}

// Stage 2 keeping the field for the adjoint: the 16 values E[ky = m][kx = n0 + i] of this
// thread's row go transposed into Ef[b][re, im][kx][ky] (fp32).  The 32 lanes of a warp hold 32
// consecutive rows, so every store instruction writes 128 contiguous bytes of one column.  (Marking
// the stores evict-first cut the contraction's operand re-reads but made the scaling pass, which
// then found none of the field in L2, slower by more: not kept.)
__device__ __forceinline__ void store_field_t(const TcArgs &a, int b, int m, int n0, const float (&er)[CW],
                                              const float (&ei)[CW]) {
    if (m >= a.M) return;
    float *o = (float *)a.out + (size_t)b * 2 * a.out_ps + (size_t)n0 * a.out_ld + m;
    if (n0 + CW <= a.N) {  // whole chunk: two running pointers, no per-column test
        float *oi = o + a.out_ps;
        const size_t ld = a.out_ld;
#pragma unroll
        for (int i = 0; i < CW; ++i) {
            *o = er[i];
            *oi = ei[i];
            o += ld;
            oi += ld;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < CW; ++i) {
        if (n0 + i < a.N) {
            o[(size_t)i * a.out_ld] = er[i];
            o[a.out_ps + (size_t)i * a.out_ld] = ei[i];
        }
    }
}

// ------------------------------------------------------------------ the kernel
template <int F, int MODE, int KIND, int PR>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapC, TcArgs a) {
    using C = Cfg<F>;
    using G = Geo<F, PR, KIND>;
    static_assert(!PR || F == FMT_F16X4, "paired: FP16 split form");
    constexpr uint32_t NBUF = (MODE == FAST) ? 2 : 1;
    // operand-writing contractions of the bf16 forms store through a staged TMA box
    constexpr bool TMA_OUT = C::TMA_STORE && (KIND == KS1 || KIND == KGE || KIND == KGT1);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stg = smem + G::STAGES * G::STAGE_BYTES;  // staged output box (TMA_OUT)
    uint64_t *bars = (uint64_t *)(stg + C::STG_BYTES);
    // bars: full[S], empty[S], tfull[2], tempty[2], drain
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * G::STAGES, tfull0 = empty0 + 8 * G::STAGES,
                   tempty0 = tfull0 + 16, drain = tempty0 + 16;
    volatile int *abort_flag = (volatile int *)(bars + 2 * G::STAGES + 5);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * G::STAGES + 6);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    pdl_wait();  // the previous kernel's outputs (operands, scales, GI) are complete from here on

    if (warp == PRODUCER_WARP) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            int u0, u1, du;
            unit_range<KIND>(a, u0, u1, du);
            for (int u = u0; u < u1 && ok; u += du) {
                int4 pc{};
                const int nj = decode_unit_jobs<KIND>(a, u, pc);
                for (int j = 0; j < nj && ok; ++j) {
                    const Job J = decode<KIND>(a, u, j, pc);
                    for (int kb = J.kb0; kb < J.kb1; ++kb, ++it) {
                        const uint32_t s = it % G::STAGES, ph = (it / G::STAGES) & 1;
                        if (!mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, a.err, 1)) {
                            ok = false;
                            break;
                        }
                        // test hook: the stage is never filled, so the MMA warp's wait for it expires
                        if (a.stall && blockIdx.x == 0 && it == 0) continue;
                        const uint32_t st = smem_u32(smem + s * G::STAGE_BYTES);
                        mbar_expect_tx(full0 + 8 * s, G::STAGE_BYTES);
                        tma_load4(st, &mapA, kb * C::KB, J.a_row, 0, J.a_batch, full0 + 8 * s);
                        tma_load4(st + G::PA * PLANE_BYTES, &mapB, kb * C::KB, J.b_row, 0, J.b_batch, full0 + 8 * s);
                    }
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                const uint32_t n = it < (uint32_t)G::STAGES ? it : (uint32_t)G::STAGES;
                for (uint32_t q = 0; q < n; ++q) {
                    const uint32_t k = it - 1 - q, s = k % G::STAGES, ph = (k / G::STAGES) & 1;
                    mbar_wait(full0 + 8 * s, ph, abort_flag, a.err, 2, true, 100000000ull);
                }
            }
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            uint32_t it = 0, jt = 0;
            bool ok = true;
            const uint32_t id_pos = idesc<F>(false), id_neg = idesc<F>(true);
            int u0, u1, du;
            unit_range<KIND>(a, u0, u1, du);
            for (int u = u0; u < u1 && ok; u += du) {
                int4 pc{};
                const int nj = decode_unit_jobs<KIND>(a, u, pc);
                for (int j = 0; j < nj && ok; ++j, ++jt) {
                    const uint32_t buf = jt % NBUF, tph = (jt / NBUF) & 1;
                    if (!mbar_wait(tempty0 + 8 * buf, tph ^ 1, abort_flag, a.err, 3)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dr = tbase + buf * 256, di = dr + 128;
                    const Job J = decode<KIND>(a, u, j, pc);
                    for (int kb = J.kb0; kb < J.kb1; ++kb, ++it) {
                        const uint32_t s = it % G::STAGES, ph = (it / G::STAGES) & 1;
                        if (!mbar_wait(full0 + 8 * s, ph, abort_flag, a.err, 4)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(smem + s * G::STAGE_BYTES), sb = sa + G::PA * PLANE_BYTES;
#pragma unroll
                        for (int ks = 0; ks < C::NKSTEP; ++ks) {
                            const uint32_t first = (kb == J.kb0 && ks == 0) ? 0u : 1u;
                            const uint32_t ko = ks * 32;
                            auto A = [&](int p) { return sdesc(sa + p * PLANE_BYTES + ko); };
                            auto Bd = [&](int p) { return sdesc(sb + p * PLANE_BYTES + ko); };
                            if constexpr (PR) {
                                // mirror-paired: matrix planes 0 hi, 1 lo of [a | b]; varying planes
                                // 0 V1 hi, 1 V1 lo, 2 V2 hi, 3 V2 lo.  Er = M.V1 with the second half
                                // of K (b . D_im) subtracted, Ei = M.V2
                                const uint32_t idr = (kb * C::KB + ks * C::KSTEP >= a.hp) ? id_neg : id_pos;
                                auto pm = [&](uint32_t d, int x, int y, uint32_t id, uint32_t acc) {
                                    if constexpr (KIND == KGE || KIND == KGP) mma<F>(d, A(y), Bd(x), id, acc);
                                    else mma<F>(d, A(x), Bd(y), id, acc);
                                };
                                if constexpr (MODE != FAST) {
                                    const uint32_t cr = tbase + 256, ci = tbase + 384;
                                    pm(dr, 0, 0, idr, first);
                                    pm(di, 0, 2, id_pos, first);
                                    pm(cr, 0, 1, idr, first);
                                    pm(cr, 1, 0, idr, 1);
                                    pm(ci, 0, 3, id_pos, first);
                                    pm(ci, 1, 2, id_pos, 1);
                                    if constexpr (MODE == SPLIT4) {
                                        pm(cr, 1, 1, idr, 1);
                                        pm(ci, 1, 3, id_pos, 1);
                                    }
                                } else {
                                    pm(dr, 0, 0, idr, first);
                                    pm(dr, 0, 1, idr, 1);
                                    pm(dr, 1, 0, idr, 1);
                                    pm(di, 0, 2, id_pos, first);
                                    pm(di, 0, 3, id_pos, 1);
                                    pm(di, 1, 2, id_pos, 1);
                                }
                            } else if constexpr (MODE != FAST) {
                                // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo; dr/di hold the hi*hi
                                // products, cr/ci the corrections
                                const uint32_t cr = tbase + 256, ci = tbase + 384;
                                mma<F>(dr, A(0), Bd(0), id_pos, first);
                                mma<F>(dr, A(2), Bd(2), id_neg, 1);
                                mma<F>(di, A(0), Bd(2), id_pos, first);
                                mma<F>(di, A(2), Bd(0), id_pos, 1);
                                mma<F>(cr, A(0), Bd(1), id_pos, first);
                                mma<F>(cr, A(1), Bd(0), id_pos, 1);
                                mma<F>(cr, A(2), Bd(3), id_neg, 1);
                                mma<F>(cr, A(3), Bd(2), id_neg, 1);
                                mma<F>(ci, A(0), Bd(3), id_pos, first);
                                mma<F>(ci, A(1), Bd(2), id_pos, 1);
                                mma<F>(ci, A(2), Bd(1), id_pos, 1);
                                mma<F>(ci, A(3), Bd(0), id_pos, 1);
                                if constexpr (MODE == SPLIT4) {
                                    mma<F>(cr, A(1), Bd(1), id_pos, 1);
                                    mma<F>(cr, A(3), Bd(3), id_neg, 1);
                                    mma<F>(ci, A(1), Bd(3), id_pos, 1);
                                    mma<F>(ci, A(3), Bd(1), id_pos, 1);
                                }
                            } else if constexpr (C::PL == 4) {
                                // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo
                                mma<F>(dr, A(0), Bd(0), id_pos, first);
                                mma<F>(dr, A(0), Bd(1), id_pos, 1);
                                mma<F>(dr, A(1), Bd(0), id_pos, 1);
                                mma<F>(dr, A(2), Bd(2), id_neg, 1);
                                mma<F>(dr, A(2), Bd(3), id_neg, 1);
                                mma<F>(dr, A(3), Bd(2), id_neg, 1);
                                mma<F>(di, A(0), Bd(2), id_pos, first);
                                mma<F>(di, A(0), Bd(3), id_pos, 1);
                                mma<F>(di, A(1), Bd(2), id_pos, 1);
                                mma<F>(di, A(2), Bd(0), id_pos, 1);
                                mma<F>(di, A(2), Bd(1), id_pos, 1);
                                mma<F>(di, A(3), Bd(0), id_pos, 1);
                            } else {
                                // planes: 0 re, 1 im
                                mma<F>(dr, A(0), Bd(0), id_pos, first);
                                mma<F>(dr, A(1), Bd(1), id_neg, 1);
                                mma<F>(di, A(0), Bd(1), id_pos, first);
                                mma<F>(di, A(1), Bd(0), id_pos, 1);
                            }
                        }
                        mma_commit(empty0 + 8 * s);  // frees the stage once these MMAs have read it
                    }
                    if (!ok) break;
                    mma_commit(tfull0 + 8 * buf);  // accumulators ready for the epilogue
                }
            }
            // drain: every MMA issued by this thread has completed before tensor memory is freed
            mma_commit(drain);
            mbar_wait(drain, 0, abort_flag, a.err, 5, true, 100000000ull);
        }
    } else {
        // ---------------- epilogue warps 0..7: lane quarter q, column half h
        const int q = warp & 3, h = warp >> 2;
        const int row = 32 * q + lane;
        uint32_t jt = 0;
        bool ok = true;
        float acc[64];  // spectral |E|^2 accumulation (stage 2 only)
        if constexpr (KIND == KS2) {
#pragma unroll
            for (int i = 0; i < 64; ++i) acc[i] = 0.f;
        }
        int u0, u1, du;
        unit_range<KIND>(a, u0, u1, du);
        for (int u = u0; u < u1 && ok; u += du) {
            int4 pc{};
            const int nj = decode_unit_jobs<KIND>(a, u, pc);
            Job J{};
            for (int j = 0; j < nj; ++j, ++jt) {
                J = decode<KIND>(a, u, j, pc);
                const uint32_t buf = jt % NBUF, tph = (jt / NBUF) & 1;
                // every lane waits; the warp proceeds only if all lanes saw the phase,
                // so the warp-collective tensor-memory loads never diverge
                const bool got = mbar_wait(tfull0 + 8 * buf, tph, abort_flag, a.err, 6);
                bool all_got;
                if constexpr (TMA_OUT) all_got = epi_all(got);  // epilogue-wide: staging uses named barriers
                else all_got = __all_sync(0xffffffffu, got);
                if (!all_got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int m = J.m0 + row;
                float mom_x = 0.f, mom_g = 0.f;  // position moments of this row (adjoint 1^T)
                // per-job constants of the epilogues
                float w = 0.f, c = 0.f, k2 = 0.f, osc = 1.f, gmx = 0.f;
                const float *gi = nullptr;
                if constexpr (KIND == KS2) w = a.wnorm[(size_t)J.r * a.nl + J.l];
                if constexpr (KIND == KGE) {
                    const int s = J.se / a.ne, e = J.se % a.ne;
                    c = 2.f * a.wnorm[(size_t)J.r * a.nl + J.l] * slot_ptr(a.prm, PFLUX, J.r)[s];
                    gi = a.GI + ((size_t)J.r * a.ne + e) * a.nd * a.nd + min(m, a.M - 1) / a.os;
                }
                if constexpr (KIND == KGP) k2 = (float)(6.283185307179586476925286766559 / a.lam[J.l]);
                if constexpr (F == FMT_F16X4) {
                    // undo / apply the power-of-two operand scales (exact):
                    // T1t' = alpha pi sigma1 T1t, so the recomputed field carries u^-1
                    const float al = a.ascale[J.l], pi = a.pscale[2 * J.r + 1];
                    // the paired phasor carries a further 1/4
                    const float u = (PR ? 4.f : 1.f) / (al * al * pi * a.sig1);
                    if constexpr (KIND == KS1) osc = a.sig1;
                    if constexpr (KIND == KS2) w *= u * u;
                    if constexpr (KIND == KGE) c *= f16_gamma(a, J) * u;
                    if constexpr (KIND == KGT1) osc = f16_sigma2(a, J);
                    // the paired adjoint field carries gamma_b / 4
                    if constexpr (KIND == KGP) k2 /= al * al * f16_gamma(a, J) * f16_sigma2(a, J) * pi * (PR ? 0.25f : 1.f);
                }
                bool released = false;  // accumulators already handed back to the MMA warp
                if constexpr (TMA_OUT) {
                    // four rounds of one 32-column box: warp (q, h) fills rows 32q.., columns 16h..,
                    // one thread stores the box; rows and columns past the tensor are clipped by TMA
                    const int zb = (KIND == KS1) ? J.b : J.z;
                    // adjoint field: the 16 GI factors of a round's columns ky (detector row ky / os),
                    // loaded one round ahead so their latency overlaps the previous round
                    float gcur[CW], gnxt[CW];
                    auto gi_round = [&](int t, float (&g)[CW]) {
                        const int n0 = J.n0 + 32 * t + 16 * h;
                        int brow = n0 / a.os, rem = n0 - brow * a.os;
                        const int bmax = (a.N - 1) / a.os;
#pragma unroll
                        for (int i = 0; i < CW; ++i) {
                            g[i] = __ldg(gi + (size_t)min(brow, bmax) * a.nd);
                            if (++rem == a.os) {
                                rem = 0;
                                ++brow;
                            }
                        }
                    };
                    if constexpr (KIND == KGE) gi_round(0, gcur);
                    // one accumulator buffer (stage 1 with hi*hi apart): the last kHold rounds are
                    // loaded together and the accumulators handed back to the MMA warp before their work
                    constexpr bool kEarly = (KIND == KS1 && MODE != FAST);
                    auto ld_round = [&](int t, float (&er)[CW], float (&ei)[CW]) {
                        const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + buf * 256 + 32 * t + 16 * h;
                        tmem_ld16(ta, er);
                        tmem_ld16(ta + 128, ei);
                        if constexpr (MODE != FAST) {
                            float tt[CW];
                            tmem_ld16(ta + 256, tt);
#pragma unroll
                            for (int i = 0; i < CW; ++i) er[i] += tt[i];
                            tmem_ld16(ta + 384, tt);
#pragma unroll
                            for (int i = 0; i < CW; ++i) ei[i] += tt[i];
                        }
                    };
                    // rounds loaded before the hand-back: three in the FP16 form (stage 1 0.617 ->
                    // 0.589 ms at the calibration size, with 80 bytes of spills), two in the BF16 forms
                    constexpr int kHold = (F == FMT_F16X4) ? 3 : 2;
                    float pre_r[kHold][CW], pre_i[kHold][CW];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (J.n0 + 32 * t >= a.out_ld) break;  // uniform over the epilogue warps
                        const int c0 = 32 * t + 16 * h;
                        if constexpr (KIND == KGE) {
                            if (t < 3) gi_round(t + 1, gnxt);
                        }
                        float er[CW], ei[CW];
                        if (kEarly && t >= 4 - kHold) {
                            if (t == 4 - kHold) {
#pragma unroll
                                for (int k = 0; k < kHold; ++k)
                                    if (J.n0 + 32 * (t + k) < a.out_ld) ld_round(t + k, pre_r[k], pre_i[k]);
                                tc_fence_before();
                                __syncwarp();
                                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
                                released = true;
                            }
#pragma unroll
                            for (int i = 0; i < CW; ++i) {
                                er[i] = pre_r[t - (4 - kHold)][i];
                                ei[i] = pre_i[t - (4 - kHold)][i];
                            }
                        } else {
                            ld_round(t, er, ei);
                        }
                        if constexpr (KIND == KGE) {
#pragma unroll
                            for (int i = 0; i < CW; ++i) {
                                const float f = c * gcur[i];
                                er[i] *= f;
                                ei[i] *= f;
                                gcur[i] = gnxt[i];
                            }
                            if constexpr (F == FMT_F16X4) {
#pragma unroll
                                for (int i = 0; i < CW; ++i) gmx = fmaxf(gmx, fmaxf(fabsf(er[i]), fabsf(ei[i])));
                            }
                        } else if constexpr (F == FMT_F16X4) {
#pragma unroll
                            for (int i = 0; i < CW; ++i) {
                                er[i] *= osc;
                                ei[i] *= osc;
                            }
                        }
                        if constexpr (PR && (KIND == KS1 || KIND == KGT1)) {
                            // paired stage 1 (adjoint 2^T): columns hp.. hold the products of the
                            // y-differences (kx-differences), stored as (Im, Re)
                            if (J.n0 + c0 >= a.hp) {
#pragma unroll
                                for (int i = 0; i < CW; ++i) {
                                    const float t = er[i];
                                    er[i] = ei[i];
                                    ei[i] = t;
                                }
                            }
                        }
                        // the previous round's box may be refilled once the TMA has read it; that
                        // read overlapped this round's tensor-memory loads and scaling
                        if (threadIdx.x == 0) bulk_wait_read0();
                        epi_bar();
                        bool staged = false;
                        if constexpr (KIND == KS1 && F == FMT_BF16X4) {
                            if (a.sr) {
                                const int n = J.n0 + c0;
                                stage_row16_sr(stg, row, h, er, ei, ((size_t)(J.b % a.B) * a.M + m) * a.out_ld + n,
                                               a.sr ^ 0xcc9e2d51u);
                                staged = true;
                            }
                        }
                        if constexpr ((KIND == KGE || KIND == KGT1) && F == FMT_BF16X2) {
                            if (a.sr) {  // BF16x3sa adjoint: stochastically rounded hi parts only
                                const int n = J.n0 + c0;
                                stage_row16_hi_sr(stg, row, h, er, ei, ((size_t)(J.b % a.B) * a.M + m) * a.out_ld + n,
                                                  a.sr);
                                staged = true;
                            }
                        }
                        if (!staged) stage_row16<F>(stg, row, h, er, ei);
                        fence_async_smem();
                        epi_bar();
                        if (threadIdx.x == 0) {
                            tma_store4(&mapC, smem_u32(stg), J.n0 + 32 * t, J.m0, 0, zb);
                            bulk_commit();
                        }
                    }
                }
                if constexpr (KIND == KS2) {
                    // stage 2: four 16-column chunks of this warp's accumulator half; chunks 2 and 3 are
                    // loaded together and the accumulators handed back to the MMA warp before their
                    // |E|^2 sums and field stores (a third chunk held would spill far more registers
                    // than the 44 bytes this costs at the 168-register limit of ten warps)
                    auto ld_chunk = [&](int cc, float (&er)[CW], float (&ei)[CW]) {
                        const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + buf * 256 + 64 * h + CW * cc;
                        tmem_ld16(ta, er);
                        tmem_ld16(ta + 128, ei);
                        if constexpr (MODE != FAST) {
                            float t[CW];
                            tmem_ld16(ta + 256, t);
#pragma unroll
                            for (int i = 0; i < CW; ++i) er[i] += t[i];
                            tmem_ld16(ta + 384, t);
#pragma unroll
                            for (int i = 0; i < CW; ++i) ei[i] += t[i];
                        }
                    };
                    auto use_chunk = [&](int cc, const float (&er)[CW], const float (&ei)[CW]) {
#pragma unroll
                        for (int i = 0; i < CW; ++i)
                            acc[CW * cc + i] = fmaf(w, er[i] * er[i] + ei[i] * ei[i], acc[CW * cc + i]);
                        // the field kept for the adjoint (FP16 form: the raw accumulators; the scaling
                        // pass applies the operand scales)
                        if constexpr (F == FMT_BF16X4 || F == FMT_F16X4 || F == FMT_TF32X4) {
                            if (a.out) store_field_t(a, J.b, m, J.n0 + 64 * h + CW * cc, er, ei);
                        }
                    };
                    float er[CW], ei[CW], er2[CW], ei2[CW];
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        ld_chunk(cc, er, ei);
                        use_chunk(cc, er, ei);
                    }
                    ld_chunk(2, er2, ei2);
                    ld_chunk(3, er, ei);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
                    use_chunk(2, er2, ei2);
                    use_chunk(3, er, ei);
                }
#pragma unroll
                for (int cc = 0; cc < ((TMA_OUT || KIND == KS2) ? 0 : 64 / CW); ++cc) {
                    const int c0 = 64 * h + CW * cc;
                    const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + buf * 256 + c0;
                    float er[CW], ei[CW];
                    tmem_ld16(ta, er);
                    tmem_ld16(ta + 128, ei);
                    if constexpr (MODE != FAST) {
                        float t[CW];
                        tmem_ld16(ta + 256, t);
#pragma unroll
                        for (int i = 0; i < CW; ++i) er[i] += t[i];
                        tmem_ld16(ta + 384, t);
#pragma unroll
                        for (int i = 0; i < CW; ++i) ei[i] += t[i];
                    }
                    const int n0 = J.n0 + c0;
                    const int nvalid = min(CW, a.N - n0);
                    if constexpr (KIND == KS2) {
                    } else {
                        if (m < a.M && nvalid > 0) {
                            if constexpr (KIND == KGE) {
                                // rows kx, columns ky: scale by 2 w_l F_s GI[e][bin(ky, kx)]; the
                                // detector row of column ky = n0 + i advances without divisions
                                int brow = n0 / a.os, rem = n0 - brow * a.os;
                                const int bmax = (a.N - 1) / a.os;
#pragma unroll
                                for (int i = 0; i < CW; ++i) {
                                    const float f = c * gi[min(brow, bmax) * a.nd];
                                    er[i] *= f;
                                    ei[i] *= f;
                                    if (++rem == a.os) {
                                        rem = 0;
                                        ++brow;
                                    }
                                }
                            }
                            if constexpr (KIND == KGP) {
                                // rows ny, columns nx: gphi = (2 pi / lambda) Im(G_P conj P)
                                const size_t pps = (size_t)a.ni * a.ldi;
                                float *o = a.gphi + ((size_t)J.b * a.ksplit + J.split) * a.ni * a.ni + (size_t)m * a.ni +
                                           n0;
                                float pr[CW], pi[CW], gv[CW];
                                if constexpr (F == FMT_BF16X2) {
                                    if (a.p4) {  // BF16x3sa: the phasor is a four-plane split, read hi + lo
                                        const char *pb = (const char *)a.P + (size_t)J.b * 4 * pps * 2;
                                        load_row<FMT_BF16X4>(pb, pps, (size_t)m * a.ldi + n0, pr, pi, nvalid);
                                    } else {
                                        const char *pb = (const char *)a.P + (size_t)J.b * C::PL * pps * C::ES;
                                        load_row<F>(pb, pps, (size_t)m * a.ldi + n0, pr, pi, nvalid);
                                    }
                                } else {
                                    const char *pb = (const char *)a.P + (size_t)J.b * C::PL * pps * C::ES;
                                    load_row<F>(pb, pps, (size_t)m * a.ldi + n0, pr, pi, nvalid);
                                }
#pragma unroll
                                for (int i = 0; i < CW; ++i) {
                                    gv[i] = (i < nvalid) ? k2 * (ei[i] * pr[i] - er[i] * pi[i]) : 0.f;
                                    // position moments of this row: sum g x_n and sum g
                                    mom_x = fmaf(gv[i], ((float)(n0 + i) - a.cNf) * a.dxf, mom_x);
                                    mom_g += gv[i];
                                }
                                if (nvalid == CW && (a.ni & 3) == 0) {
#pragma unroll
                                    for (int qq = 0; qq < CW / 4; ++qq)
                                        *(float4 *)(o + 4 * qq) =
                                            make_float4(gv[4 * qq], gv[4 * qq + 1], gv[4 * qq + 2], gv[4 * qq + 3]);
                                } else {
#pragma unroll
                                    for (int i = 0; i < CW; ++i)
                                        if (i < nvalid) o[i] = gv[i];
                                }
                            } else {
                                const int zb = (KIND == KS1) ? J.b : J.z;
                                char *ob = (char *)a.out + (size_t)zb * C::PL * a.out_ps * C::ES;
                                store_row<F>(ob, a.out_ps, (size_t)m * a.out_ld + n0, er, ei, nvalid);
                            }
                        }
                    }
                }
                if (KIND != KS2 && !released) {  // stage 2 handed its accumulators back above
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
                }
                if constexpr (F == FMT_F16X4 && KIND == KGE) {
                    // max |GEt'| of this PSF (non-negative floats order as their bits)
                    if (!(gmx < 3.0e38f)) gmx = 3.0e38f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, o));
                    if (lane == 0) atomicMax(a.gmax + J.b, __float_as_uint(gmx));
                }
                if constexpr (KIND == KGP) {
                    // per-warp position moments of this tile, reduced in a fixed order:
                    // mom[entry][tile][warp] = (sum g x_n, sum g y_n), entry = PSF x K split
                    float sy = (m < a.M) ? mom_g * (((float)m - a.cNf) * a.dxf) : 0.f;
                    float sx = mom_x;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        sx += __shfl_xor_sync(0xffffffffu, sx, o);
                        sy += __shfl_xor_sync(0xffffffffu, sy, o);
                    }
                    if (lane == 0) {
                        const int tile = (J.m0 / BM) * a.tn + J.n0 / BN;
                        const size_t ent = (size_t)J.b * a.ksplit + J.split;
                        float2 *dst = (float2 *)a.mom + ((ent * a.tm * a.tn + tile) * EPI_WARPS + warp);
                        *dst = make_float2(sx, sy);
                    }
                }
            }
            if (!ok) break;
            if constexpr (KIND == KS2) {
                // the piece's partial sum goes to its plane; the last piece of a segment
                // also clears the planes the split left unwritten for this tile
                const int m = J.m0 + row, rse = pc.x / (a.tm * a.tn);
                const int plane = pc.w & 0xffff, zf = pc.w >> 16;
                if (m < a.M) {
                    const size_t pl = (size_t)a.no * a.no;
                    float *o = a.Is + ((size_t)plane * a.Rnse + rse) * pl + (size_t)m * a.no + J.n0 + 64 * h;
                    const int nv = a.N - (J.n0 + 64 * h);
                    if (nv >= 64 && (a.no & 3) == 0) {
#pragma unroll
                        for (int i = 0; i < 64; i += 4)
                            *(float4 *)(o + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
                        for (int q = zf; q < a.G; ++q) {
                            float *z = o + (size_t)(q - plane) * a.Rnse * pl;
#pragma unroll
                            for (int i = 0; i < 64; i += 4) *(float4 *)(z + i) = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 64; ++i)
                            if (i < nv) o[i] = acc[i];
                        for (int q = zf; q < a.G; ++q) {
                            float *z = o + (size_t)(q - plane) * a.Rnse * pl;
                            for (int i = 0; i < 64 && i < nv; ++i) z[i] = 0.f;
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 64; ++i) acc[i] = 0.f;
            }
        }
        if constexpr (TMA_OUT) {
            if (threadIdx.x == 0) bulk_wait0();  // the last boxes have reached global memory
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    // looked up once per process (thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return nullptr;
    }();
    return fn;
}

// Tensor map of an operand: 4-D {k, row, plane, batch}, box 128 rows x 64 bytes x all
// planes.  hi_view: the planes re_hi and im_hi (0 and 2) of a four-plane split operand,
// as a two-plane tensor (plane stride doubled).
bool make_map(dlx_plan *p, Operand &o, std::string *why, bool hi_view = false) {
    auto enc = get_encoder();
    if (!enc) {
        *why = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    const int es = p->esz, PL = hi_view ? 2 : o.planes;
    const cuuint64_t plane = (cuuint64_t)o.rows * o.ld * es;
    cuuint64_t dims[4] = {(cuuint64_t)o.ld, (cuuint64_t)o.rows, (cuuint64_t)PL, (cuuint64_t)o.batch};
    cuuint64_t strides[3] = {(cuuint64_t)o.ld * es, (hi_view ? 2 : 1) * plane, (cuuint64_t)o.planes * plane};
    cuuint32_t box[4] = {(cuuint32_t)(64 / es), 128u, (cuuint32_t)PL, 1u};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMapDataType dt = (p->fmt == FMT_TF32X4)  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : (p->fmt == FMT_F16X4) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(hi_view ? &o.tmap_hi : &o.tmap, dt, 4, o.ptr, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

template <int F, int MODE, int KIND, int PR = 0>
cudaError_t launch(dlx_plan *p, const Operand &A, const Operand &B, const Operand *Cout, TcArgs &a,
                   cudaStream_t st) {
    // the shared-memory attribute is a property of the kernel on each device: set once per device
    static std::atomic<uint64_t> attr_set{0};
    const uint64_t dev_bit = 1ull << (p->device & 63);
    if (!(attr_set.load(std::memory_order_acquire) & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<F, MODE, KIND, PR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Geo<F, PR, KIND>::SMEM);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(dev_bit, std::memory_order_release);
    }
    a.err = p->err;
    a.nl = p->nl;
    a.nse = p->nse;
    a.B = p->B;
    a.ne = p->ne;
    a.nd = p->nd;
    a.os = p->os;
    a.ni = p->ni;
    a.no = p->no;
    a.ldi = p->ldi;
    a.ldo = p->ldo;
    a.G = p->G;
    a.wnorm = p->wnorm;
    a.lam = p->lam_d;
    a.ascale = p->ascale;
    a.pscale = p->pscale;
    a.sig1 = inv_pow2_ceil((float)p->ni);
    a.qmax = p->qmax;
    a.gmax = p->gmax;
    a.sr = (KIND == KS1) ? p->sr
           : (p->adj1 && KIND == KGE) ? p->sr ^ 0x85ebca77u
           : (p->adj1 && KIND == KGT1) ? p->sr ^ 0xc2b2ae3du
                                       : 0u;
    a.p4 = (p->adj1 && KIND == KGP) ? 1 : 0;
    a.hp = PR ? ((KIND == KGT1 || KIND == KGP) ? p->hpo : p->hp) : 0;
    a.tm = (a.M + BM - 1) / BM;
    a.tn = (a.N + BN - 1) / BN;
    a.KB = Cfg<F>::KB;
    if (a.ksplit < 1) a.ksplit = 1;
    if (a.units <= 0) return cudaSuccess;
    a.stall = p->inject == 1 ? 1 : 0;
    p->inject = 0;
    const int grid = a.grid > 0 ? a.grid : std::min(a.units, p->sm_count);
    static const int cls_of[5] = {KC_STAGE1, KC_STAGE2, KC_ADJ_FIELD, KC_ADJ2, KC_ADJ1};
    KScope ks(p, cls_of[KIND], 1, st);
    return launch_pdl(k_tc_gemm<F, MODE, KIND, PR>, dim3(grid), dim3(NTHREADS), Geo<F, PR, KIND>::SMEM, st, A.tmap,
                      B.tmap, Cout ? Cout->tmap : A.tmap, a);
}

// MODE1 / MODE2: accumulation modes of stage 1 and stage 2
template <int F, int MODE1, int MODE2, int PR>
cudaError_t forward_impl(dlx_plan *p, int R, cudaStream_t st) {
    TcArgs a{};
    // stage 1: T1t[b] = A(l) . P[b]^T   (M = No rows kx, N = Ni cols ny, K = Ni); mirror-paired:
    // the paired phasor's 2 hp rows and K = 2 hp, written in the paired layout (pair_layout)
    a.M = p->no;
    a.N = PR ? 2 * p->hp : p->ni;
    a.K = PR ? 2 * p->hp : p->ni;
    a.out = p->T1t.ptr;
    a.out_ld = p->T1t.ld;
    a.out_ps = (size_t)p->no * p->T1t.ld;
    a.units = R * p->B * ((a.M + BM - 1) / BM) * ((a.N + BN - 1) / BN);
    cudaError_t e = launch<F, MODE1, KS1, PR>(p, p->amat, PR ? p->Pp : p->P, &p->T1t, a, st);
    if (e != cudaSuccess) return e;
    // stage 2 + intensity: Is[g][rse] = sum_l w |A(l) . T1t[b]^T|^2  (M = N = No, K = Ni; paired 2 hp)
    TcArgs c{};
    c.M = p->no;
    c.N = p->no;
    c.K = PR ? 2 * p->hp : p->ni;
    c.Is = p->Is;
    c.Rnse = R * p->nse;
    const dlx_plan::S2Split &sp = p->s2[R - 1];
    c.s2off = p->s2_table + sp.off;
    c.s2pc = (const int4 *)(p->s2_table + sp.pcs);
    c.grid = sp.nct;
    c.units = sp.npieces;
    if (p->keep_field) {  // E of every PSF, transposed: Ef[b][re, im][kx][ky]
        c.out = p->Ef;
        c.out_ld = p->ldo;
        c.out_ps = (size_t)p->no * p->ldo;
    }
    return launch<F, MODE2, KS2, PR>(p, p->amat, p->T1t, nullptr, c, st);
}

template <int F>
cudaError_t adjoint_impl(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st) {
    const int tmo = (p->no + BM - 1) / BM, tmi = (p->ni + BM - 1) / BM;
    TcArgs a{};
    // recomputed field and dL/dE: GEt[z][kx][ky] = 2 w F GI o (T1t[b] . A(l)^T)
    a.M = p->no;
    a.N = p->no;
    a.K = p->paired ? 2 * p->hp : p->ni;
    a.b0 = b0;
    a.prm = prm;
    a.GI = p->GI;
    a.out = p->GEt.ptr;
    a.out_ld = p->ldo;
    a.out_ps = (size_t)p->no * p->ldo;
    a.units = nb * tmo * tmo;
    // BF16x3sa: the recomputed field contracts the stochastic hi planes of T1t and A only
    Operand T1 = p->T1t, Am = p->amat;
    if (p->adj1) {
        T1.tmap = p->T1t.tmap_hi;
        Am.tmap = p->amat.tmap_hi;
    }
    // the field kept by stage 2 (split forms) is scaled and split; otherwise it is recomputed
    cudaError_t e;
    if (p->keep_field) {
        e = launch_field_scale(p, prm, b0, nb, st);
    } else if constexpr (F == FMT_F16X4) {
        e = p->paired ? launch<F, FAST, KGE, 1>(p, T1, Am, &p->GEt, a, st) : launch<F, FAST, KGE>(p, T1, Am, &p->GEt, a, st);
    } else {
        e = launch<F, FAST, KGE>(p, T1, Am, &p->GEt, a, st);
    }
    if (e != cudaSuccess) return e;
    // adjoint stage 2^T: GT1[z][ny][kx] = AH(l) . GEt[z]^T   (M = Ni, N = No, K = No); mirror-paired
    // (FP16 form with the field kept): N = K = 2 hpo, the paired field from the scaling pass
    constexpr int PA = (F == FMT_F16X4) ? 1 : 0;
    const bool pa = PA && p->padj;
    if (p->padj && !p->keep_field) return cudaErrorInvalidValue;  // the paired operand comes from the pass
    TcArgs b{};
    b.M = p->ni;
    b.N = pa ? 2 * p->hpo : p->no;
    b.K = pa ? 2 * p->hpo : p->no;
    b.b0 = b0;
    b.prm = prm;
    b.out = p->GT1.ptr;
    b.out_ld = p->GT1.ld;
    b.out_ps = (size_t)p->ni * p->GT1.ld;
    b.units = nb * tmi * ((b.N + BN - 1) / BN);
    e = pa ? launch<F, FAST, KGT1, PA>(p, p->amatH, p->GEt, &p->GT1, b, st)
           : launch<F, FAST, KGT1>(p, p->amatH, p->GEt, &p->GT1, b, st);
    if (e != cudaSuccess) return e;
    // adjoint stage 1^T + phase gradient: gphi[b][split] = (2 pi/lambda) Im((GT1[z] . AH(l)^T) conj P[b]),
    // the K = No contraction split in gsplit parts (their gphi planes are summed by the reductions)
    TcArgs c{};
    c.M = p->ni;
    c.N = p->ni;
    c.K = pa ? 2 * p->hpo : p->no;
    c.b0 = b0;
    c.prm = prm;
    c.P = p->P.ptr;
    c.gphi = p->gphi;
    c.mom = p->mom;
    c.dxf = (float)p->dx;
    c.cNf = 0.5f * (float)(p->ni - 1);
    c.ksplit = p->gsplit;
    c.units = nb * tmi * tmi * p->gsplit;
    return pa ? launch<F, FAST, KGP, PA>(p, p->GT1, p->amatH, nullptr, c, st)
              : launch<F, FAST, KGP>(p, p->GT1, p->amatH, nullptr, c, st);
}

}  // namespace

int tc_supported(const dlx_plan *p, std::string *why) {
    if (p->fmt == FMT_F32) {
        *why = "FP32 form runs on CUDA cores";
        return 0;
    }
    return 1;
}

int tc_make_maps(dlx_plan *p, std::string *why) {
    bool ok = make_map(p, p->amat, why) && make_map(p, p->amatH, why) && make_map(p, p->P, why) &&
              make_map(p, p->T1t, why) && make_map(p, p->GEt, why) && make_map(p, p->GT1, why);
    if (ok && p->adj1) ok = make_map(p, p->amat, why, true) && make_map(p, p->T1t, why, true);
    if (ok && p->paired) ok = make_map(p, p->Pp, why);
    return ok;
}

cudaError_t tc_forward(dlx_plan *p, int R, cudaStream_t st) {
    switch (p->fmt) {
        case FMT_BF16X4:
            if (p->prec == DLX_BF16X4) return forward_impl<FMT_BF16X4, SPLIT4, SPLIT4, 0>(p, R, st);
            // BF16x3 (stochastic split): stage 1 double-buffers its accumulators up to a 256-long
            // contraction; beyond, hi*hi accumulates apart there too (its truncation grows with K)
            return p->ni <= 256 ? forward_impl<FMT_BF16X4, FAST, SPLIT3, 0>(p, R, st)
                                : forward_impl<FMT_BF16X4, SPLIT3, SPLIT3, 0>(p, R, st);
        case FMT_BF16X2: return forward_impl<FMT_BF16X2, FAST, FAST, 0>(p, R, st);
        case FMT_TF32X4: return forward_impl<FMT_TF32X4, SPLIT3, SPLIT3, 0>(p, R, st);
        case FMT_F16X4: return forward_impl<FMT_F16X4, SPLIT3, SPLIT3, 1>(p, R, st);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t tc_adjoint_chunk(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st) {
    switch (p->fmt) {
        case FMT_BF16X4:
            // BF16x3sa: one product per real product on the stochastic hi parts (two-plane kernels)
            return p->adj1 ? adjoint_impl<FMT_BF16X2>(p, prm, b0, nb, st) : adjoint_impl<FMT_BF16X4>(p, prm, b0, nb, st);
        case FMT_BF16X2: return adjoint_impl<FMT_BF16X2>(p, prm, b0, nb, st);
        case FMT_TF32X4: return adjoint_impl<FMT_TF32X4>(p, prm, b0, nb, st);
        case FMT_F16X4: return adjoint_impl<FMT_F16X4>(p, prm, b0, nb, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace dlx
