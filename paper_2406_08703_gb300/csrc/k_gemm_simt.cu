// FP32 CUDA-core form of the four MFT contractions (Sec. 3, two-sided MFT).
//
// Every contraction is C[m][n] = sum_k A[m][k] B[n][k] over complex operands
// stored as re/im FP32 planes with both operands contiguous in k.  A 256-thread
// block owns a 64 x 64 output tile; each thread holds a 4 x 4 complex
// register tile (rows 4 ty + i, columns 4 tx + j), read per k from shared memory
// as four 16-byte vectors (re and im of its four rows and of its four columns),
// so that 64 FMAs take four shared-memory loads and sixteen threads store 64
// contiguous floats of a row.  Operand tiles of 16 k are staged in shared memory
// transposed to [k][row] (rows padded to 68 words: 16-byte aligned, and the
// transposing stores spread over the banks).  The epilogues are the same as in
// the tensor-core form.
#include "dlx_common.cuh"

namespace dlx {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

constexpr int PAD = 4;  // row padding of the staged tiles (keeps float4 reads aligned)

struct SimtSmem {
    __align__(16) float ar[BK][BM + PAD];
    __align__(16) float ai[BK][BM + PAD];
    __align__(16) float br[BK][BN + PAD];
    __align__(16) float bi[BK][BN + PAD];
};

// Accumulates the tile (m0, n0) of A . B^T into (cr, ci).  PF: load the next k-block from
// global memory while the current one is multiplied (16 more registers; measured faster for
// stage 1 and the adjoint 2^T and 1^T, no faster for the recomputed field, and stage 2, which
// also holds the spectral sum, spilled with it).
template <bool PF>
__device__ __forceinline__ void simt_tile(const float *__restrict__ A, size_t a_ps, int lda, int M,
                                          const float *__restrict__ Bm, size_t b_ps, int ldb, int N, int K, int m0,
                                          int n0, float (&cr)[4][4], float (&ci)[4][4], SimtSmem &sm) {
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    constexpr int NR = (BM * BK) / NT;  // staged elements per thread and array
    // the next k-block's operands are loaded into registers while the current one is
    // multiplied out of shared memory
    float vr[NR], vi[NR], wr[NR], wi[NR];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int idx = tid + r * NT, row = idx / BK, kk = idx % BK, gk = k0 + kk;
            const int gm = m0 + row, gn = n0 + row;
            vr[r] = vi[r] = wr[r] = wi[r] = 0.f;
            if (gm < M && gk < K) {
                const size_t o = (size_t)gm * lda + gk;
                vr[r] = A[o];
                vi[r] = A[a_ps + o];
            }
            if (gn < N && gk < K) {
                const size_t o = (size_t)gn * ldb + gk;
                wr[r] = Bm[o];
                wi[r] = Bm[b_ps + o];
            }
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        if (!PF && k0 > 0) fetch(k0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int idx = tid + r * NT, row = idx / BK, kk = idx % BK;
            sm.ar[kk][row] = vr[r];
            sm.ai[kk][row] = vi[r];
            sm.br[kk][row] = wr[r];
            sm.bi[kk][row] = wi[r];
        }
        __syncthreads();
        if (PF && k0 + BK < K) fetch(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 ar4 = *(const float4 *)&sm.ar[kk][4 * ty], ai4 = *(const float4 *)&sm.ai[kk][4 * ty];
            const float4 br4 = *(const float4 *)&sm.br[kk][4 * tx], bi4 = *(const float4 *)&sm.bi[kk][4 * tx];
            const float a_r[4] = {ar4.x, ar4.y, ar4.z, ar4.w}, a_i[4] = {ai4.x, ai4.y, ai4.z, ai4.w};
            const float b_r[4] = {br4.x, br4.y, br4.z, br4.w}, b_i[4] = {bi4.x, bi4.y, bi4.z, bi4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cr[i][j] = fmaf(a_r[i], b_r[j], cr[i][j]);
                    cr[i][j] = fmaf(-a_i[i], b_i[j], cr[i][j]);
                    ci[i][j] = fmaf(a_r[i], b_i[j], ci[i][j]);
                    ci[i][j] = fmaf(a_i[i], b_r[j], ci[i][j]);
                }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void zero(float (&c)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
}

// Stage 1: T1t[b][kx][ny] = sum_nx A(l)[kx][nx] P[b][ny][nx].
__global__ void __launch_bounds__(NT, 2) k_simt_stage1(const float *amat, const float *P, float *T1t, int ni, int no,
                                                    int ldi, int nse, int B) {
    __shared__ SimtSmem sm;
    const int b = blockIdx.z, l = (b % B) / nse, m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    float cr[4][4], ci[4][4];
    zero(cr);
    zero(ci);
    const size_t aps = (size_t)no * ldi, pps = (size_t)ni * ldi;
    simt_tile<true>(amat + (size_t)l * 2 * aps, aps, ldi, no, P + (size_t)b * 2 * pps, pps, ldi, ni, ni, m0, n0, cr, ci, sm);
    float *out = T1t + (size_t)b * 2 * aps;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int m = m0 + 4 * ty + i, n = n0 + 4 * tx + j;
            if (m < no && n < ni) {
                out[(size_t)m * ldi + n] = cr[i][j];
                out[aps + (size_t)m * ldi + n] = ci[i][j];
            }
        }
}

// Stage 2 + intensity: Is[g][r nse + se][ky][kx] = sum_{l in group g} w_l |sum_ny A(l)[ky][ny] T1t[b][kx][ny]|^2.
// With Ef, every PSF's field is also kept for the adjoint: Ef[b][re, im][ky][kx] (rows of ldo).
__global__ void __launch_bounds__(NT, 2) k_simt_stage2(const float *amat, const float *T1t, const float *wnorm, float *Is,
                                                    int ni, int no, int ldi, int nse, int nl, int G, int tiles_n,
                                                    int B, float *Ef, int ldo) {
    __shared__ SimtSmem sm;
    const int rse = blockIdx.y, r = rse / nse, se = rse % nse, g = blockIdx.z;
    const int m0 = (blockIdx.x / tiles_n) * BM, n0 = (blockIdx.x % tiles_n) * BN;
    const int l0 = (int)((long)g * nl / G), l1 = (int)((long)(g + 1) * nl / G);
    const size_t aps = (size_t)no * ldi;
    float acc[4][4];
    zero(acc);
    for (int l = l0; l < l1; ++l) {
        float cr[4][4], ci[4][4];
        zero(cr);
        zero(ci);
        const int b = r * B + l * nse + se;
        simt_tile<false>(amat + (size_t)l * 2 * aps, aps, ldi, no, T1t + (size_t)b * 2 * aps, aps, ldi, no, ni, m0, n0, cr,
                  ci, sm);
        const float w = wnorm[(size_t)r * nl + l];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(w, cr[i][j] * cr[i][j] + ci[i][j] * ci[i][j], acc[i][j]);
        if (Ef) {
            const size_t eps = (size_t)no * ldo;
            float *er = Ef + (size_t)b * 2 * eps, *ei = er + eps;
            const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = m0 + 4 * ty + i, n = n0 + 4 * tx;
                if (m >= no) continue;
                if (n + 3 < no && (ldo & 3) == 0) {
                    *(float4 *)(er + (size_t)m * ldo + n) = make_float4(cr[i][0], cr[i][1], cr[i][2], cr[i][3]);
                    *(float4 *)(ei + (size_t)m * ldo + n) = make_float4(ci[i][0], ci[i][1], ci[i][2], ci[i][3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (n + j < no) {
                            er[(size_t)m * ldo + n + j] = cr[i][j];
                            ei[(size_t)m * ldo + n + j] = ci[i][j];
                        }
                }
            }
        }
    }
    float *out = Is + ((size_t)g * gridDim.y + rse) * no * no;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int m = m0 + 4 * ty + i, n = n0 + 4 * tx + j;
            if (m < no && n < no) out[(size_t)m * no + n] = acc[i][j];
        }
}

// Adjoint, recomputed field: E^T[kx][ky] = sum_ny T1t[b][kx][ny] A(l)[ky][ny];
// GEt[z][kx][ky] = 2 w_l F_s GI[e][bin(ky,kx)] E^T[kx][ky]  (dL/dRe E + i dL/dIm E).
__global__ void __launch_bounds__(NT, 2) k_simt_grad_field(const float *amat, const float *T1t, const float *wnorm,
                                                        DevParams prm, const float *GI, float *GEt, int ni, int no,
                                                        int ldi, int ldo, int nl, int nse, int ne, int nd, int os,
                                                        int B, int b0, int tiles_n) {
    __shared__ SimtSmem sm;
    const int z = blockIdx.y, b = b0 + z, r = b / B, bl = b % B, l = bl / nse, se = bl % nse, s = se / ne,
              e = se % ne;
    const int m0 = (blockIdx.x / tiles_n) * BM, n0 = (blockIdx.x % tiles_n) * BN;
    const size_t aps = (size_t)no * ldi;
    float cr[4][4], ci[4][4];
    zero(cr);
    zero(ci);
    simt_tile<false>(T1t + (size_t)b * 2 * aps, aps, ldi, no, amat + (size_t)l * 2 * aps, aps, ldi, no, ni, m0, n0, cr, ci,
              sm);
    const float c = 2.f * wnorm[(size_t)r * nl + l] * slot_ptr(prm, PFLUX, r)[s];
    const float *gi = GI + ((size_t)r * ne + e) * nd * nd;
    const size_t gps = (size_t)no * ldo;
    float *out = GEt + (size_t)z * 2 * gps;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int kx = m0 + 4 * ty + i, ky = n0 + 4 * tx + j;
            if (kx < no && ky < no) {
                float f = c * gi[(ky / os) * nd + kx / os];
                out[(size_t)kx * ldo + ky] = f * cr[i][j];
                out[gps + (size_t)kx * ldo + ky] = f * ci[i][j];
            }
        }
}

// Adjoint field from the field stage 2 kept: GEt[z][kx][ky] = 2 w_l F_s GI[e][bin(ky,kx)] E[ky][kx],
// the values k_simt_grad_field computes, transposed through 32 x 32 tiles in shared memory.
__global__ void k_simt_field_scale(const float *__restrict__ Ef, const float *__restrict__ wnorm, DevParams prm,
                                   const float *__restrict__ GI, float *GEt, int no, int ldo, int nl, int nse, int ne,
                                   int nd, int os, int B, int b0) {
    __shared__ float tr[32][33], ti[32][33];
    const int z = blockIdx.z, b = b0 + z, r = b / B, bl = b % B, l = bl / nse, se = bl % nse, s = se / ne,
              e = se % ne;
    const int kx0 = blockIdx.x * 32, ky0 = blockIdx.y * 32;
    const size_t ps = (size_t)no * ldo;
    const float *er = Ef + (size_t)b * 2 * ps, *ei = er + ps;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ky = ky0 + threadIdx.y + 8 * k, kx = kx0 + threadIdx.x;
        if (ky < no && kx < no) {
            tr[threadIdx.y + 8 * k][threadIdx.x] = er[(size_t)ky * ldo + kx];
            ti[threadIdx.y + 8 * k][threadIdx.x] = ei[(size_t)ky * ldo + kx];
        }
    }
    __syncthreads();
    const float c = 2.f * wnorm[(size_t)r * nl + l] * slot_ptr(prm, PFLUX, r)[s];
    const float *gi = GI + ((size_t)r * ne + e) * nd * nd;
    float *gr = GEt + (size_t)z * 2 * ps, *gim = gr + ps;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int kx = kx0 + threadIdx.y + 8 * k, ky = ky0 + threadIdx.x;
        if (kx < no && ky < no) {
            const float f = c * gi[(ky / os) * nd + kx / os];
            gr[(size_t)kx * ldo + ky] = f * tr[threadIdx.x][threadIdx.y + 8 * k];
            gim[(size_t)kx * ldo + ky] = f * ti[threadIdx.x][threadIdx.y + 8 * k];
        }
    }
}

// Adjoint stage 2^T: GT1[z][ny][kx] = sum_ky AH(l)[ny][ky] GEt[z][kx][ky].
__global__ void __launch_bounds__(NT, 2) k_simt_adj2(const float *amatH, const float *GEt, float *GT1, int ni, int no,
                                                  int ldo, int nse, int B, int b0) {
    __shared__ SimtSmem sm;
    const int z = blockIdx.z, b = b0 + z, l = (b % B) / nse, m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const size_t hps = (size_t)ni * ldo, gps = (size_t)no * ldo;
    float cr[4][4], ci[4][4];
    zero(cr);
    zero(ci);
    simt_tile<true>(amatH + (size_t)l * 2 * hps, hps, ldo, ni, GEt + (size_t)z * 2 * gps, gps, ldo, no, no, m0, n0, cr, ci,
              sm);
    float *out = GT1 + (size_t)z * 2 * hps;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int m = m0 + 4 * ty + i, n = n0 + 4 * tx + j;
            if (m < ni && n < no) {
                out[(size_t)m * ldo + n] = cr[i][j];
                out[hps + (size_t)m * ldo + n] = ci[i][j];
            }
        }
}

// Adjoint stage 1^T + phase gradient: G_P[ny][nx] = sum_kx GT1[z][ny][kx] AH(l)[nx][kx];
// gphi[b][ny][nx] = (2 pi / lambda_l) Im(G_P conj(P[b][ny][nx])).
__global__ void __launch_bounds__(NT, 2) k_simt_adj1(const float *amatH, const float *GT1, const float *P,
                                                  const double *lam, float *gphi, int ni, int no, int ldi, int ldo,
                                                  int nse, int B, int b0) {
    __shared__ SimtSmem sm;
    const int z = blockIdx.z, b = b0 + z, l = (b % B) / nse, m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const size_t hps = (size_t)ni * ldo, pps = (size_t)ni * ldi;
    float cr[4][4], ci[4][4];
    zero(cr);
    zero(ci);
    simt_tile<true>(GT1 + (size_t)z * 2 * hps, hps, ldo, ni, amatH + (size_t)l * 2 * hps, hps, ldo, ni, no, m0, n0, cr, ci,
              sm);
    const float k2 = (float)(6.283185307179586476925286766559 / lam[l]);
    const float *pb = P + (size_t)b * 2 * pps;
    float *out = gphi + (size_t)b * ni * ni;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int ny = m0 + 4 * ty + i, nx = n0 + 4 * tx + j;
            if (ny < ni && nx < ni) {
                float pr = pb[(size_t)ny * ldi + nx], pi = pb[pps + (size_t)ny * ldi + nx];
                out[(size_t)ny * ni + nx] = k2 * (ci[i][j] * pr - cr[i][j] * pi);
            }
        }
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t simt_forward(dlx_plan *p, int R, cudaStream_t st) {
    const float *amat = (const float *)p->amat.ptr;
    dim3 g1(cdiv(p->no, BM), cdiv(p->ni, BN), R * p->B);
    {
    KScope ks(p, KC_STAGE1, 1, st);
    k_simt_stage1<<<g1, NT, 0, st>>>(amat, (const float *)p->P.ptr, (float *)p->T1t.ptr, p->ni, p->no, p->ldi, p->nse,
                                     p->B);
    }
    int tn = cdiv(p->no, BN);
    dim3 g2(cdiv(p->no, BM) * tn, R * p->nse, p->G);
    KScope ks(p, KC_STAGE2, 1, st);
    k_simt_stage2<<<g2, NT, 0, st>>>(amat, (const float *)p->T1t.ptr, p->wnorm, p->Is, p->ni, p->no, p->ldi, p->nse,
                                     p->nl, p->G, tn, p->B, p->keep_field ? (float *)p->Ef : nullptr, p->ldo);
    return cudaGetLastError();
}

cudaError_t simt_adjoint_chunk(dlx_plan *p, const DevParams &prm, int b0, int nb, cudaStream_t st) {
    const float *amat = (const float *)p->amat.ptr, *amatH = (const float *)p->amatH.ptr;
    int tn = cdiv(p->no, BN);
    dim3 ge(cdiv(p->no, BM) * tn, nb);
    if (p->keep_field) {  // the field stage 2 kept, scaled and transposed
        KScope ks(p, KC_FIELD_SCALE, 1, st);
        const int t32 = cdiv(p->no, 32);
        k_simt_field_scale<<<dim3(t32, t32, nb), dim3(32, 8), 0, st>>>((const float *)p->Ef, p->wnorm, prm, p->GI,
                                                                       (float *)p->GEt.ptr, p->no, p->ldo, p->nl,
                                                                       p->nse, p->ne, p->nd, p->os, p->B, b0);
    } else {
        KScope ks(p, KC_ADJ_FIELD, 1, st);
        k_simt_grad_field<<<ge, NT, 0, st>>>(amat, (const float *)p->T1t.ptr, p->wnorm, prm, p->GI,
                                             (float *)p->GEt.ptr, p->ni, p->no, p->ldi, p->ldo, p->nl, p->nse, p->ne,
                                             p->nd, p->os, p->B, b0, tn);
    }
    dim3 g2(cdiv(p->ni, BM), cdiv(p->no, BN), nb);
    {
    KScope ks(p, KC_ADJ2, 1, st);
    k_simt_adj2<<<g2, NT, 0, st>>>(amatH, (const float *)p->GEt.ptr, (float *)p->GT1.ptr, p->ni, p->no, p->ldo, p->nse,
                                   p->B, b0);
    }
    dim3 g1(cdiv(p->ni, BM), cdiv(p->ni, BN), nb);
    KScope ks(p, KC_ADJ1, 1, st);
    k_simt_adj1<<<g1, NT, 0, st>>>(amatH, (const float *)p->GT1.ptr, (const float *)p->P.ptr, p->lam_d, p->gphi, p->ni,
                                   p->no, p->ldi, p->ldo, p->nse, p->B, b0);
    return cudaGetLastError();
}

}  // namespace dlx
