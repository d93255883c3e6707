// extend_df.cu -- the extension of f on cut leaves (Sections 3.2, 4.1) in the
// mixed form: double-float arithmetic (df32.cuh) plus one exact-slice table
// GEMM.  The steps are those of the FP64 kernel k_extend, spread over four
// launches so that no CTA streams a whole cut leaf's operators alone:
//
//   1. k_ext_coeff_df  c = A_I^+ f_I, one warp per row of A_I^+ (a GEMV
//                      streaming the per-leaf pseudo-inverses from HBM);
//   2. table GEMM      A_{X_Sbar,G} c at all Kbar^2 grid points of every cut
//                      leaf at once (one universal table, gemm_frag.cu);
//   3. k_ext_alpha_df  one CTA per cut leaf: the grid takes the data at
//                      interior points; its Chebyshev coefficients, truncated
//                      to m + n < Kbar;
//   4. k_ext_eval_df   one CTA per target leaf (the cut leaf itself and each
//                      leaf of its extension list): the expansion at the
//                      target's nodes.
//
// Operators are stored as double-float pairs; data enter and leave as FP64.
// Relative errors stay near 2^-47 times the extension's conditioning (step 2,
// a five-slice pass: 2^-40 of its own terms), at or below the 39 bits of the
// leaf values that the mixed form's slices keep.
#include <cmath>

#include "bulk.cuh"
#include "dev_common.cuh"
#include "df32.cuh"
#include "ext.cuh"
#include "slice_math.cuh"

namespace vpx {

__device__ inline df32 ld_df(const float2 *p) {
    const float2 v = *p;
    return df32{v.x, v.y};
}

__device__ inline float2 st_df(df32 v) { return make_float2(v.hi, v.lo); }

// grid (ncut * nrb, rhs), 256 threads: warp w of block b computes row
// k = (b % nrb) * 8 + w of c for cut leaf b / nrb.  The block's 8 rows of
// A_I^+ (contiguous, rows padded to an even length) arrive by one TMA bulk copy
// while the threads split f_I.
__global__ void __launch_bounds__(256) k_ext_coeff_df(ExtArgs a, int nrb, double *cbuf, int64_t ldc, int *status) {
    pdl_entry();
    extern __shared__ __align__(16) float2 csm[];
    __shared__ __align__(8) uint64_t s_bar;
    const int c = blockIdx.x / nrb, rb = blockIdx.x % nrb, rhs = blockIdx.y;
    const int nI = a.n_interior[c], NG = a.NG, nIp = (nI + 1) & ~1;
    const int k0 = rb * 8, nrow = min(8, NG - k0);
    float2 *Ps = csm, *fI = csm + 8 * (size_t)nIp;
    if (threadIdx.x == 0) {
        bulk_bar_init(&s_bar);
        const uint32_t bytes = (uint32_t)(nrow * nIp * sizeof(float2));
        bulk_expect(&s_bar, bytes);
        bulk_copy(Ps, a.pinv_df + a.pinv_df_off[c] + (size_t)k0 * nIp, bytes, &s_bar);
    }
    const double *f = a.f + rhs * a.ldf + a.stencil_off[c];
    for (int i = threadIdx.x; i < nI; i += blockDim.x) fI[i] = st_df(df_split_bits(f[i]));
    __syncthreads();
    if (!__syncthreads_and(bulk_wait(&s_bar, 0))) {
        if (threadIdx.x == 0) set_status(status, VPX_ERR_TIMEOUT);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= nrow) return;
    const float2 *P = Ps + (size_t)warp * nIp;
    df32 s{0.f, 0.f};
    for (int i = lane; i < nI; i += 32) df_mac(s, ld_df(P + i), ld_df(fI + i));
    s = df_warp_sum(s);
    if (lane == 0) cbuf[rhs * ldc + (int64_t)c * NG + k0 + warp] = df_value(s);
}

// The truncated Chebyshev coefficients of a cut leaf's Kbar x Kbar grid
// values F (shared memory, [by][ax]): T1[m][by] = sum_ax C[m][ax] F[by][ax],
// then alpha[m][n] = sum_by T1[m][by] C[n][by] for m + n < Kbar (zero beyond),
// into al (global).  All threads of the block; T1 is shared scratch.
__device__ inline void ext_alpha_from_grid(const float2 *C, const float2 *F, float2 *T1, int Kb, float2 *al) {
    const int Kb2 = Kb * Kb;
    for (int e = threadIdx.x; e < Kb2; e += blockDim.x) {
        const int m = e / Kb, by = e % Kb;
        df32 s{0.f, 0.f};
        for (int ax = 0; ax < Kb; ++ax) df_mac(s, ld_df(C + m * Kb + ax), ld_df(F + by * Kb + ax));
        T1[m * Kb + by] = st_df(df_norm(s));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Kb2; e += blockDim.x) {
        const int m = e / Kb, n = e % Kb;
        df32 s{0.f, 0.f};
        if (m + n < Kb)
            for (int by = 0; by < Kb; ++by) df_mac(s, ld_df(T1 + m * Kb + by), ld_df(C + n * Kb + by));
        al[e] = st_df(df_norm(s));
    }
}

constexpr int kExtPerThread = 4;   // grid points per thread in k_ext_alpha_df (Kbar^2 <= 1024)

// grid (cut leaves, rhs), 256 threads: the grid takes the data at interior
// points and A_{X_Sbar,G} c elsewhere; alpha = C F C^T truncated to m + n < Kbar
__global__ void __launch_bounds__(256) k_ext_alpha_df(ExtArgs a, const double *Fall, int64_t ldF, float2 *alpha,
                                                     int64_t lda, int *status) {
    pdl_entry();
    extern __shared__ __align__(16) float2 smf[];
    __shared__ __align__(8) uint64_t s_bar;
    const int c = blockIdx.x, rhs = blockIdx.y;
    const int Kb = a.Kbar, Kb2 = Kb * Kb, Kb2p = (Kb2 + 1) & ~1;   // Kb2p: 16-byte multiple
    float2 *C = smf;               // Kb2   Chebyshev transform [m][ax]
    float2 *F = C + Kb2p;          // Kb2   grid values [by][ax]
    float2 *T1 = F + Kb2p;         // Kb2   [m][by]
    if (threadIdx.x == 0) {
        bulk_bar_init(&s_bar);
        bulk_expect(&s_bar, (uint32_t)(Kb2p * sizeof(float2)));
        bulk_copy(C, a.cheb_df, (uint32_t)(Kb2p * sizeof(float2)), &s_bar);
    }
    const double *f = a.f + rhs * a.ldf + a.stencil_off[c];
    const int32_t *gs = a.grid_src + (size_t)c * Kb2;
    const double *Fc = Fall + rhs * ldF + (int64_t)c * Kb2;
    // independent loads first (source index and grid value), then the data
    int src[kExtPerThread];
    double v[kExtPerThread];
#pragma unroll
    for (int q = 0; q < kExtPerThread; ++q) {
        const int g = threadIdx.x + q * blockDim.x;
        src[q] = (g < Kb2) ? gs[g] : -1;
        v[q] = (g < Kb2) ? Fc[g] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kExtPerThread; ++q)
        if (src[q] >= 0) v[q] = f[src[q]];
#pragma unroll
    for (int q = 0; q < kExtPerThread; ++q) {
        const int g = threadIdx.x + q * blockDim.x;
        if (g < Kb2) F[g] = st_df(df_split_bits(v[q]));
    }
    __syncthreads();
    if (!__syncthreads_and(bulk_wait(&s_bar, 0))) {
        if (threadIdx.x == 0) set_status(status, VPX_ERR_TIMEOUT);
        return;
    }
    ext_alpha_from_grid(C, F, T1, Kb, alpha + rhs * lda + (int64_t)c * Kb2p);
}

// grid (targets, rhs), 256 threads: the truncated expansion of the target's
// cut leaf at the target's K x K nodes (interior nodes of the cut leaf itself
// keep the data).  geo[t] = (x offset, y offset, node scale) of the target in
// the coordinates of the cut leaf's Sbar, and whether it is the cut leaf.
__global__ void __launch_bounds__(256) k_ext_eval_df(ExtArgs a, const int32_t *tgt_cut, const int32_t *tgt_leaf,
                                                    const ExtTgtGeo *geo, const float2 *alpha, int64_t lda,
                                                    int *status) {
    pdl_entry();
    extern __shared__ __align__(16) float2 smf[];
    __shared__ __align__(8) uint64_t s_bar;
    const int t = blockIdx.x, rhs = blockIdx.y;
    const int c = tgt_cut[t], tl = tgt_leaf[t];
    const ExtTgtGeo gt = geo[t];
    const int K = a.K, KK = K * K, Kb = a.Kbar, Kb2p = (Kb * Kb + 1) & ~1;
    float2 *al = smf;              // Kb2   alpha[m][n]
    float2 *Tx = al + Kb2p;        // K*Kb  T_m at the target x nodes
    float2 *Ty = Tx + K * Kb;      // K*Kb
    float2 *G = Ty + K * Kb;       // Kb*K
    if (threadIdx.x == 0) {
        bulk_bar_init(&s_bar);
        bulk_expect(&s_bar, (uint32_t)(Kb2p * sizeof(float2)));
        bulk_copy(al, alpha + rhs * lda + (int64_t)c * Kb2p, (uint32_t)(Kb2p * sizeof(float2)), &s_bar);
    }
    // Chebyshev values at the target coordinates (FP64 recurrence, 2K x Kb values)
    for (int e = threadIdx.x; e < 2 * K; e += blockDim.x) {
        const int i = e % K;
        const double z = ((e < K) ? gt.ox : gt.oy) + gt.sc * a.tnodes[i];
        float2 *T = (e < K) ? Tx + i * Kb : Ty + i * Kb;
        double tp = 1.0, tc = z;   // T_{m-1}, T_m
        T[0] = st_df(df_split(1.0));
        if (Kb > 1) T[1] = st_df(df_split_bits(z));
        for (int m = 2; m < Kb; ++m) {
            const double tn = 2.0 * z * tc - tp;
            tp = tc;
            tc = tn;
            T[m] = st_df(df_split_bits(tn));
        }
    }
    __syncthreads();
    if (!__syncthreads_and(bulk_wait(&s_bar, 0))) {
        if (threadIdx.x == 0) set_status(status, VPX_ERR_TIMEOUT);
        return;
    }
    // G[n][ax] = sum_m alpha[m][n] Tx[ax][m]
    for (int e = threadIdx.x; e < Kb * K; e += blockDim.x) {
        const int n = e / K, ax = e % K;
        df32 s{0.f, 0.f};
        for (int m = 0; m + n < Kb; ++m) df_mac(s, ld_df(al + m * Kb + n), ld_df(Tx + ax * Kb + m));
        G[n * K + ax] = st_df(df_norm(s));
    }
    __syncthreads();
    const double *f = a.f + rhs * a.ldf + a.stencil_off[c];
    double *out = a.fe + rhs * a.ldfe + (int64_t)tl * KK;
    const int32_t *ns = a.node_src + (size_t)c * KK;
    const bool self = gt.self != 0.0;
    double val = 0.0;   // node threadIdx.x (KK <= 256 = blockDim.x)
    for (int j = threadIdx.x; j < KK; j += blockDim.x) {
        const int ax = j % K, by = j / K;
        const int src = self ? ns[j] : -1;
        if (src >= 0) {
            val = f[src];
        } else {
            df32 s{0.f, 0.f};
            for (int n = 0; n < Kb; ++n) df_mac(s, ld_df(Ty + by * Kb + n), ld_df(G + n * K + ax));
            val = df_to_f64_scaled(df_norm(s), 0);
        }
        out[j] = val;
    }
    if (a.fe_sl) {   // the leaf's exact slices, as the potential's passes read them
        __shared__ uint64_t s_mb[8];
        uint64_t m = slice_abs_bits(val);   // 0 for the threads past the leaf's KK nodes
        for (int o = 16; o; o >>= 1) {
            const uint64_t t = (uint64_t)__shfl_xor_sync(0xffffffffu, (long long)m, o);
            m = t > m ? t : m;
        }
        if ((threadIdx.x & 31) == 0) s_mb[threadIdx.x >> 5] = m;
        __syncthreads();
        uint64_t mx = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = s_mb[w] > mx ? s_mb[w] : mx;
        const int e = slice_expo_of_bits(mx);
        const int j = threadIdx.x;
        if (j < a.kpad) {
            uint16_t d[kSlicesS];
            slice_digits(slice_fixed_point(j < KK ? val : 0.0, e), d);
            uint16_t *o = a.fe_sl + ((size_t)rhs * a.n_leaves + tl) * kSlicesS * a.kpad + j;
#pragma unroll
            for (int k = 0; k < kSlicesS; ++k) o[(size_t)k * a.kpad] = d[k];
        }
        if (j == 0) a.fe_ex[(size_t)rhs * a.n_leaves + tl] = e;
    }
}

static size_t kb2p(int Kb) { return ((size_t)Kb * Kb + 1) & ~(size_t)1; }
static size_t alpha_smem(int Kb) { return sizeof(float2) * 3 * kb2p(Kb); }
static size_t eval_smem(int K, int Kb) { return sizeof(float2) * (kb2p(Kb) + 3 * (size_t)K * Kb); }


static size_t coeff_smem(int max_interior) {
    const size_t nIp = (size_t)(max_interior + 1) & ~(size_t)1;
    return sizeof(float2) * (8 * nIp + nIp);
}

void extend_df_prepare(int max_interior, int K, int Kbar) {
    if (coeff_smem(max_interior) > 48 * 1024)
        VPX_CUDA(cudaFuncSetAttribute(k_ext_coeff_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)coeff_smem(max_interior)));
    if (alpha_smem(Kbar) > 48 * 1024)
        VPX_CUDA(cudaFuncSetAttribute(k_ext_alpha_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)alpha_smem(Kbar)));
    if (eval_smem(K, Kbar) > 48 * 1024)
        VPX_CUDA(cudaFuncSetAttribute(k_ext_eval_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)eval_smem(K, Kbar)));
}

void launch_ext_coeff_df(const ExtArgs &a, int ncut, int max_interior, int nrhs, double *cbuf, int64_t ldc,
                         int *status, cudaStream_t s) {
    const int nrb = (a.NG + 7) / 8;
    launch_pdl(k_ext_coeff_df, dim3(ncut * nrb, nrhs), dim3(256), coeff_smem(max_interior), s, a, nrb, cbuf, ldc, status);
    VPX_LAUNCH("k_ext_coeff_df");
}

void launch_ext_eval_df(const ExtArgs &a, int ncut, int n_tgt, const int32_t *tgt_cut, const int32_t *tgt_leaf,
                        const ExtTgtGeo *geo, const double *Fall, int64_t ldF, float2 *alpha, int nrhs, int *status,
                        cudaStream_t s) {
    if (a.Kbar * a.Kbar > kExtPerThread * 256) fail(VPX_ERR_ARG, "extension grid larger than one block covers");
    const int64_t lda = (int64_t)ncut * kb2p(a.Kbar);
    launch_pdl(k_ext_alpha_df, dim3(ncut, nrhs), dim3(256), alpha_smem(a.Kbar), s, a, Fall, ldF, alpha, lda, status);
    VPX_LAUNCH("k_ext_alpha_df");
    launch_pdl(k_ext_eval_df, dim3(n_tgt, nrhs), dim3(256), eval_smem(a.K, a.Kbar), s, a, tgt_cut, tgt_leaf, geo, alpha, lda,
                                                                          status);
    VPX_LAUNCH("k_ext_eval_df");
}

}  // namespace vpx
