// gemm_rows.cu -- the grouped table GEMM (gemm.cuh) in double-float
// arithmetic (df32.cuh) on the fp32 pipes, for passes too small to amortise
// the exact-slice engines' slicing and recombination: the level-by-level
// chains M2M and L2L of the mixed form, whose every level holds a few hundred
// 2(p+1) x 2(p+1) products.
//
// One CTA takes R_NPB pairs of one table; a thread owns one table row and a
// share of the inner index, with one double-float accumulator per pair
// (independent chains).  About 48 significant bits, more than the 42-bit
// slices of the tensor-core passes keep.
#include "dev_common.cuh"
#include "df32.cuh"
#include "gemm.cuh"

namespace vpx {

constexpr int R_NPB = kRowsTileN;
constexpr int R_KG = 4;   // k groups per CTA (rows <= 96)

// CTA = R_KG groups of ceil32(M) threads; group g sums k = g, g + R_KG, ...
// for its row; the table and the source vectors are staged in shared memory
// first (one coalesced copy each), the group partials are added at the end.
__global__ void __launch_bounds__(384) k_gemm_rows_df(int M, int Kd, int kg, const float2 *tT, const GTile *tiles,
                                                      const GPair *pairs, const double *vbase, int64_t vld,
                                                      int vstride, double *out, int64_t ldo, int add) {
    extern __shared__ __align__(16) float2 rsm[];   // table [Kd][M], vectors [R_NPB][Kd], partials [kg][R_NPB][M]
    __shared__ GPair s_pr[R_NPB];
    __shared__ int s_e[R_NPB];
    float2 *Ts = rsm, *vsm = Ts + (size_t)Kd * M, *part = vsm + R_NPB * Kd;
    const GTile tile = tiles[blockIdx.x];
    const int rhs = blockIdx.y, nt = blockDim.x;
    const float2 *T = tT + (size_t)tile.tab * Kd * M;
    for (int c = threadIdx.x; c < Kd * M; c += nt) Ts[c] = __ldg(T + c);
    if (threadIdx.x < R_NPB) {
        const GPair pr = (threadIdx.x < tile.count) ? pairs[tile.first + threadIdx.x] : GPair{0, 0, -1, 0.0};
        s_pr[threadIdx.x] = pr;
        int e = 0;
        frexp(pr.scale, &e);   // the pair scales of these passes are powers of two: 2^(e-1)
        s_e[threadIdx.x] = e - 1;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < R_NPB * Kd; c += nt) {
        const int n = c / Kd, k = c % Kd;
        const double x = (n < tile.count) ? vbase[rhs * vld + (int64_t)s_pr[n].src * vstride + k] : 0.0;
        const df32 v = df_split_bits(x);
        vsm[c] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    const int mr = nt / kg, g = threadIdx.x / mr, i = threadIdx.x % mr;
    if (i < M) {
        df32 acc[R_NPB];
#pragma unroll
        for (int j = 0; j < R_NPB; ++j) acc[j] = df32{0.f, 0.f};
        for (int k = g; k < Kd; k += kg) {
            const float2 t = Ts[(size_t)k * M + i];
#pragma unroll
            for (int j = 0; j < R_NPB; ++j) {
                const float2 v = vsm[j * Kd + k];
                df_mac(acc[j], df32{t.x, t.y}, df32{v.x, v.y});
            }
        }
#pragma unroll
        for (int j = 0; j < R_NPB; ++j) {
            const df32 a = df_norm(acc[j]);
            part[((size_t)g * R_NPB + j) * M + i] = make_float2(a.hi, a.lo);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < R_NPB * M; c += nt) {
        const int j = c / M, r = c % M;
        if (j >= tile.count) continue;
        df32 s{0.f, 0.f};
        for (int q = 0; q < kg; ++q) {
            const float2 v = part[((size_t)q * R_NPB + j) * M + r];
            s = df_add(s, df32{v.x, v.y});
        }
        const double val = df_to_f64_scaled(s, s_e[j]);
        double *o = out + rhs * ldo + s_pr[j].dst + r;
        if (add) atomicAdd(o, val);
        else *o = val;
    }
}

static size_t rows_smem(int M, int Kd, int kg) {
    return sizeof(float2) * ((size_t)Kd * M + (size_t)R_NPB * Kd + (size_t)kg * R_NPB * M);
}

void gemm_rows_prepare(const GemmPass &g) {
    const int kg = g.M <= 96 ? R_KG : 1;
    const size_t smem = rows_smem(g.M, g.Kd, kg);
    if (smem > 48 * 1024)
        VPX_CUDA(cudaFuncSetAttribute(k_gemm_rows_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}

void gemm_rows_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s) {
    if (g.n_tiles_r == 0) return;
    const int kg = g.M <= 96 ? R_KG : 1;
    const int threads = (g.M + 31) / 32 * 32 * kg;
    if (threads > 384) fail(VPX_ERR_ARG, "row engine: too many table rows");
    k_gemm_rows_df<<<dim3(g.n_tiles_r, nrhs), threads, rows_smem(g.M, g.Kd, kg), (cudaStream_t)s>>>(
        g.M, g.Kd, kg, reinterpret_cast<const float2 *>(g.tdfT), g.tiles_r, g.pairs, vs.base, vs.ld, vs.stride, out,
        ldo, g.add);
    VPX_LAUNCH("k_gemm_rows_df");
}

}  // namespace vpx
