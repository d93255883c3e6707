// gemm_rows.cu -- the grouped table GEMM (gemm.cuh) in double-float
// arithmetic (df32.cuh) on the fp32 pipes, for passes too small to amortise
// the exact-slice engines' slicing and recombination: the level-by-level
// chains M2M and L2L of the mixed form, whose every level holds a few hundred
// 2(p+1) x 2(p+1) products.
//
// One CTA takes NPB pairs of one table (1, or 8 on passes of many pairs, where
// one table copy per pair would dominate the traffic); a thread owns one table
// row and a share of the inner index, with one double-float accumulator per
// pair (independent chains).  About 48 significant bits, more than the 39-bit
// slices of the tensor-core passes keep.  Every pair is summed in the same
// order for either NPB.
#include "bulk.cuh"
#include "dev_common.cuh"
#include "df32.cuh"
#include "gemm.cuh"

namespace vpx {

static_assert(kRowsTileN == 1, "the row engine's one-pair tiles");
constexpr int R_KG = 4;              // k groups per CTA (rows <= 96)
constexpr int R_WIDE = 8;            // pairs per CTA on passes of many pairs
constexpr int R_WIDE_FROM = 1024;    // pairs from which a pass takes R_WIDE pairs per CTA

// CTA = R_KG groups of ceil32(M) threads; group g sums k = g, g + R_KG, ...
// for its row.  The table arrives in shared memory by one TMA bulk copy while
// the threads fetch and split the source vector; the group partials are added
// at the end.
template <int NPB>
__global__ void __launch_bounds__(384) k_gemm_rows_df(int M, int Kd, int kg, int64_t tstride, const float2 *tT,
                                                      const GTile *tiles, const GPair *pairs, const double *vbase,
                                                      int64_t vld, int vstride, double *out, int64_t ldo, int add,
                                                      int *status) {
    pdl_entry();
    extern __shared__ __align__(16) float2 rsm[];   // table [Kd][M], vectors [NPB][Kd], partials [kg][NPB][M]
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_e[NPB];
    __shared__ int64_t s_dst[NPB];
    float2 *Ts = rsm, *vsm = Ts + tstride, *part = vsm + NPB * Kd;
    const int rhs = blockIdx.y, nt = blockDim.x;
    const GTile tile = tiles[blockIdx.x];
    // one-pair tiles are in pair order (tile i holds pair i), so the pair loads beside its tile
    const int p0 = NPB == 1 ? (int)blockIdx.x : tile.first, np = NPB == 1 ? 1 : tile.count;
    if (threadIdx.x == 0) {
        bulk_bar_init(&s_bar);
        const uint32_t bytes = (uint32_t)(tstride * sizeof(float2));
        bulk_expect(&s_bar, bytes);
        bulk_copy(Ts, tT + (size_t)tile.tab * tstride, bytes, &s_bar);
    }
    if (threadIdx.x < NPB) {
        const int j = threadIdx.x;
        int e = 0;
        int64_t dst = -1;
        if (j < np) {
            const GPair pr = pairs[p0 + j];
            frexp(pr.scale, &e);   // the pair scales of these passes are powers of two: 2^(e-1)
            dst = pr.dst;
        }
        s_e[j] = e - 1;
        s_dst[j] = dst;
    }
    for (int c = threadIdx.x; c < NPB * Kd; c += nt) {
        const int j = c / Kd, k = c % Kd;
        double x = 0.0;
        if (j < np) x = vbase[rhs * vld + (int64_t)pairs[p0 + j].src * vstride + k];
        const df32 v = df_split_bits(x);
        vsm[c] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (!__syncthreads_and(bulk_wait(&s_bar, 0))) {   // every thread leaves together on a timeout
        if (threadIdx.x == 0) set_status(status, VPX_ERR_TIMEOUT);
        return;
    }
    const int mr = nt / kg, g = threadIdx.x / mr, i = threadIdx.x % mr;
    if (i < M) {
        df32 acc[NPB];
#pragma unroll
        for (int j = 0; j < NPB; ++j) acc[j] = df32{0.f, 0.f};
        for (int k = g; k < Kd; k += kg) {
            const float2 t = Ts[(size_t)k * M + i];
#pragma unroll
            for (int j = 0; j < NPB; ++j) {
                const float2 v = vsm[j * Kd + k];
                df_mac(acc[j], df32{t.x, t.y}, df32{v.x, v.y});
            }
        }
#pragma unroll
        for (int j = 0; j < NPB; ++j) {
            const df32 a = df_norm(acc[j]);
            part[((size_t)g * NPB + j) * M + i] = make_float2(a.hi, a.lo);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NPB * M; c += nt) {
        const int j = c / M, r = c % M;
        if (s_dst[j] < 0) continue;
        df32 s{0.f, 0.f};
        for (int q = 0; q < kg; ++q) {
            const float2 v = part[((size_t)q * NPB + j) * M + r];
            s = df_add(s, df32{v.x, v.y});
        }
        const double val = df_to_f64_scaled(s, s_e[j]);
        double *o = out + rhs * ldo + s_dst[j] + r;
        if (add) atomicAdd(o, val);
        else *o = val;
    }
}

static int64_t rows_tstride(int M, int Kd) { return ((int64_t)Kd * M + 1) / 2 * 2; }   // 16-byte multiple

static size_t rows_smem(int M, int Kd, int kg, int npb) {
    return sizeof(float2) * ((size_t)rows_tstride(M, Kd) + (size_t)npb * Kd + (size_t)kg * npb * M);
}

// the pass's 8-pair tiles (the fragment engine keeps one list of 8 and one of 32)
static const GTile *rows_wide_tiles(const GemmPass &g, int &n) {
    n = g.np_f == R_WIDE ? g.n_tiles_f : g.np_f_alt == R_WIDE ? g.n_tiles_f_alt : 0;
    return g.np_f == R_WIDE ? g.tiles_f : g.np_f_alt == R_WIDE ? g.tiles_f_alt : nullptr;
}

void gemm_rows_prepare(const GemmPass &g) {
    const int kg = g.M <= 96 ? R_KG : 1;
    const size_t s1 = rows_smem(g.M, g.Kd, kg, 1), s8 = rows_smem(g.M, g.Kd, kg, R_WIDE);
    if (s1 > 48 * 1024)
        VPX_CUDA(cudaFuncSetAttribute(k_gemm_rows_df<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1));
    if (s8 > 48 * 1024)
        VPX_CUDA(cudaFuncSetAttribute(k_gemm_rows_df<R_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s8));
}

void gemm_rows_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s) {
    if (g.n_tiles_r == 0) return;
    const int kg = g.M <= 96 ? R_KG : 1;
    const int threads = (g.M + 31) / 32 * 32 * kg;
    if (threads > 384) fail(VPX_ERR_ARG, "row engine: too many table rows");
    if (g.n_tiles_r != g.n_pairs) fail(VPX_ERR_ARG, "row engine: one pair per tile expected");
    int n8 = 0;
    const GTile *t8 = rows_wide_tiles(g, n8);
    const float2 *tab = reinterpret_cast<const float2 *>(g.tdfT);
    if (g.n_pairs >= R_WIDE_FROM && t8 && n8 > 0)
        launch_pdl(k_gemm_rows_df<R_WIDE>, dim3(n8, nrhs), dim3(threads), rows_smem(g.M, g.Kd, kg, R_WIDE),
                   (cudaStream_t)s, g.M, g.Kd, kg, rows_tstride(g.M, g.Kd), tab, t8, g.pairs, vs.base, vs.ld,
                   vs.stride, out, ldo, g.add, g.status);
    else
        launch_pdl(k_gemm_rows_df<1>, dim3(g.n_tiles_r, nrhs), dim3(threads), rows_smem(g.M, g.Kd, kg, 1),
                   (cudaStream_t)s, g.M, g.Kd, kg, rows_tstride(g.M, g.Kd), tab, g.tiles_r, g.pairs, vs.base, vs.ld,
                   vs.stride, out, ldo, g.add, g.status);
    VPX_LAUNCH("k_gemm_rows_df");
}

}  // namespace vpx
