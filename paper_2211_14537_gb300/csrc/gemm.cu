// gemm.cu -- the two engines of the grouped table GEMM (see gemm.cuh).
//
// FP64 form: 64 x 64 output tile per CTA, 4 x 4 FP64 register tile per thread,
// 16-deep k stages in shared memory.
//
// Mixed form (exact bf16 slices): each table row i is scaled by 2^-e_i and
// split into S = 5 or 6 integer slices of 7 bits (|a_1| <= 128, |a_k| <= 64), each
// source vector likewise with its own exponent.  A product of two slices is
// an integer of at most 14 bits; for an inner dimension <= 256 the sum of all
// products of the same order d = k + l stays below 2^24, so the tensor core's
// fp32 accumulation of each order is exact.  The orders are combined in
// double-float fp32 (exact 2^-7 steps, TwoSum), converted once to FP64 and
// scaled by scale_p 2^{e_i + e_v - 14}.  Truncation error ~ 2^-7S relative to
// max|row| max|vector| (order sums stay below 8 * 2^20 < 2^24 for S <= 6).  Operand tiles are staged with cp.async (16-byte
// copies, two stages); products use mma.sync m16n8k16 bf16 -> fp32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "dev_common.cuh"
#include "gemm.cuh"
#include "slice_epilogue.cuh"

namespace vpx {

// ------------------------------------------------------------ FP64 engine

constexpr int G_M = 64, G_N = 64, G_K = 16;

__global__ void __launch_bounds__(256) k_gemm_fp64(int M, int Kd, const double *tab, const GTile *tiles,
                                                   const GPair *pairs, const double *vbase, int64_t vld,
                                                   int vstride, double *out, int64_t ldo, int add) {
    __shared__ double As[G_K][G_M + 1];
    __shared__ double Bs[G_K][G_N + 1];
    const GTile tile = tiles[blockIdx.x];
    const int m0 = blockIdx.y * G_M, rhs = blockIdx.z;
    const double *A = tab + (size_t)tile.tab * M * Kd;
    const double *V = vbase + rhs * vld;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < Kd; k0 += G_K) {
        for (int e = threadIdx.x; e < G_M * G_K; e += 256) {
            int r = e / G_K, k = e % G_K;
            As[k][r] = (m0 + r < M && k0 + k < Kd) ? A[(size_t)(m0 + r) * Kd + k0 + k] : 0.0;
        }
        for (int e = threadIdx.x; e < G_N * G_K; e += 256) {
            int n = e / G_K, k = e % G_K;
            Bs[k][n] = (n < tile.count && k0 + k < Kd)
                           ? V[(int64_t)pairs[tile.first + n].src * vstride + k0 + k]
                           : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < G_K; ++k) {
            double ar[4], br[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ar[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) br[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += ar[i] * br[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int n = tx + 16 * j;
        if (n >= tile.count) continue;
        const GPair pr = pairs[tile.first + n];
        double *o = out + rhs * ldo + pr.dst;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = m0 + ty * 4 + i;
            if (r >= M) continue;
            if (add) atomicAdd(o + r, pr.scale * acc[i][j]);
            else o[r] = pr.scale * acc[i][j];
        }
    }
}

// ------------------------------------------------------- exact bf16 engine

constexpr int X_M = 64, X_N = 64, X_K = 32;
constexpr int X_LD = X_K + 8;   // smem pitch (bf16): 80 bytes, 16-byte aligned rows, conflict-free fragments
constexpr int X_STAGE = kSlicesS * (X_M + X_N) * X_LD;   // bf16 elements per stage (room for 6 slices)

__device__ inline void cp_async16(void *smem, const void *gmem, int bytes) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ inline void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ inline void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ inline void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct SlicedArgs {
    int M, Mpad, Kpad, nvec;
    const uint16_t *tslices;   // [ntab][S][Mpad][Kpad]
    const int32_t *texpo;      // [ntab][Mpad]
    const GTile *tiles;
    const GPair *pairs;
    const uint16_t *vslices;   // [rhs][nvec][S][Kpad]
    const int32_t *vexpo;      // [rhs][nvec]
    double *out;
    int64_t ldo;
    int add;
};

// 256 threads = 8 warps: 4 along M (16 rows) x 2 along N (32 pairs).  S slices used.
template <int S>
__global__ void __launch_bounds__(256) k_gemm_sliced(SlicedArgs a) {
    extern __shared__ __align__(16) uint16_t xs[];
    const GTile tile = a.tiles[blockIdx.x];
    const int m0 = blockIdx.y * X_M, rhs = blockIdx.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2;
    const int g = lane >> 2, tq = lane & 3;
    const uint16_t *T = a.tslices + (size_t)tile.tab * kSlicesS * a.Mpad * a.Kpad;
    const uint16_t *VS = a.vslices + (size_t)rhs * a.nvec * kSlicesS * a.Kpad;
    // staging: 5 slices x 64 rows x 32 k of A and of B = 2 x 1280 16-byte chunks
    auto stage = [&](int buf, int k0) {
        uint16_t *As = xs + buf * X_STAGE;
        uint16_t *Bs = As + kSlicesS * X_M * X_LD;
        for (int c = threadIdx.x; c < S * X_M * 4; c += 256) {
            int s = c / (X_M * 4), rem = c % (X_M * 4), r = rem >> 2, q = rem & 3;
            int gr = m0 + r;
            const uint16_t *src = T + ((size_t)s * a.Mpad + (gr < a.Mpad ? gr : 0)) * a.Kpad + k0 + q * 8;
            cp_async16(As + (s * X_M + r) * X_LD + q * 8, src, gr < a.Mpad ? 16 : 0);
        }
        for (int c = threadIdx.x; c < S * X_N * 4; c += 256) {
            int s = c / (X_N * 4), rem = c % (X_N * 4), n = rem >> 2, q = rem & 3;
            bool ok = n < tile.count;
            int v = ok ? a.pairs[tile.first + n].src : 0;
            const uint16_t *src = VS + ((size_t)v * kSlicesS + s) * a.Kpad + k0 + q * 8;
            cp_async16(Bs + (s * X_N + n) * X_LD + q * 8, src, ok ? 16 : 0);
        }
        cp_async_commit();
    };
    float acc[S][4][4];
#pragma unroll
    for (int d = 0; d < S; ++d)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[d][t][r] = 0.f;
    const int nk = a.Kpad / X_K;
    stage(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) {
            stage((kt + 1) & 1, (kt + 1) * X_K);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();
        const uint16_t *As = xs + (kt & 1) * X_STAGE;
        const uint16_t *Bs = As + kSlicesS * X_M * X_LD;
#pragma unroll
        for (int kk = 0; kk < X_K; kk += 16) {
            uint32_t af[S][4];
            const int ar = wm * 16 + g;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const uint16_t *Ar = As + (s * X_M + ar) * X_LD + kk + tq * 2;
                af[s][0] = *reinterpret_cast<const uint32_t *>(Ar);
                af[s][1] = *reinterpret_cast<const uint32_t *>(Ar + 8 * X_LD);
                af[s][2] = *reinterpret_cast<const uint32_t *>(Ar + 8);
                af[s][3] = *reinterpret_cast<const uint32_t *>(Ar + 8 * X_LD + 8);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int bn = wn * 32 + t * 8 + g;
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    const uint16_t *Br = Bs + (l * X_N + bn) * X_LD + kk + tq * 2;
                    uint32_t bf[2];
                    bf[0] = *reinterpret_cast<const uint32_t *>(Br);
                    bf[1] = *reinterpret_cast<const uint32_t *>(Br + 8);
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        if (s + l < S) mma16816(acc[s + l][t], af[s], bf);
                }
            }
        }
        __syncthreads();
    }
    // epilogue
    SliceScale pscale[4][2];
    int64_t pdst[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int n = wn * 32 + t * 8 + tq * 2 + half;
            pdst[t][half] = -1;
            pscale[t][half] = SliceScale{0.f, 0.f, 0};
            if (n < tile.count) {
                const GPair pr = a.pairs[tile.first + n];
                pscale[t][half] = slice_pair_scale(pr.scale, a.vexpo[(size_t)rhs * a.nvec + pr.src] - 2 * kSliceBitsB);
                pdst[t][half] = rhs * a.ldo + pr.dst;
            }
        }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int i = m0 + wm * 16 + g + rr * 8;
        if (i >= a.M) continue;
        const int row_e = a.texpo[(size_t)tile.tab * a.Mpad + i];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (pdst[t][half] < 0) continue;
                float acc_d[S], hi, lo;
#pragma unroll
                for (int d = 0; d < S; ++d) acc_d[d] = acc[d][t][rr * 2 + half];
                slice_recombine<S>(acc_d, hi, lo);
                const double val = slice_output(hi, lo, pscale[t][half], row_e);
                double *o = a.out + pdst[t][half] + i;
                if (a.add) atomicAdd(o, val);
                else *o = val;
            }
    }
}

// ------------------------------------------------------------ slicing

__device__ __host__ inline int slice_expo(double amax) {
    if (!(amax > 0.0)) return 0;
    int e;
    frexp(amax, &e);
    return e;
}

// one block per (vector, rhs): exponent of max|v| and S slices over Kpad (zero padded)
__global__ void k_slice_vec(const double *vbase, int64_t vld, int vstride, int first, int Kd, int Kpad, int nvec,
                            uint16_t *slices, int32_t *expo) {
    const int v = first + blockIdx.x, rhs = blockIdx.y;
    const double *x = vbase + rhs * vld + (int64_t)v * vstride;
    __shared__ double s_max[32];
    double m = 0.0;
    for (int j = threadIdx.x; j < Kd; j += blockDim.x) m = fmax(m, fabs(x[j]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, s_max[w]);
        s_max[0] = mm;
    }
    __syncthreads();
    const int e = slice_expo(s_max[0]);
    __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(slices) + ((size_t)rhs * nvec + v) * kSlicesS * Kpad;
    for (int j = threadIdx.x; j < Kpad; j += blockDim.x) {
        double y = (j < Kd) ? ldexp(x[j], -e) : 0.0;
        for (int k = 0; k < kSlicesS; ++k) {
            y = ldexp(y, kSliceBitsB);
            double q = rint(y);
            y -= q;
            out[(size_t)k * Kpad + j] = __double2bfloat16(q);
        }
    }
    if (threadIdx.x == 0) expo[(size_t)rhs * nvec + v] = e;
}

// ------------------------------------------------------------------ host

void gemm_pass_set_pairs(GemmPass &g, std::vector<std::pair<int, GPair>> &tagged) {
    std::stable_sort(tagged.begin(), tagged.end(),
                     [](const std::pair<int, GPair> &x, const std::pair<int, GPair> &y) { return x.first < y.first; });
    std::vector<GPair> pr;
    std::vector<GTile> tl;
    size_t i = 0;
    while (i < tagged.size()) {
        size_t j = i;
        while (j < tagged.size() && tagged[j].first == tagged[i].first) ++j;
        for (size_t k = i; k < j; k += kGemmTileN)
            tl.push_back({tagged[i].first, (int32_t)(pr.size() + (k - i)), (int32_t)std::min<size_t>(kGemmTileN, j - k), 0});
        for (size_t k = i; k < j; ++k) pr.push_back(tagged[k].second);
        i = j;
    }
    g.h_pairs = pr;
    g.n_pairs = (int)pr.size();
    g.n_tiles = (int)tl.size();
    g.pairs = dev_upload(pr);
    g.tiles = dev_upload(tl);
}

static uint16_t bf16_bits_exact(double q) {
    // q is an integer with |q| <= 256: exact in bf16
    __nv_bfloat16 b = __double2bfloat16(q);
    return *reinterpret_cast<uint16_t *>(&b);
}

void gemm_pass_upload_tables(GemmPass &g, const std::vector<double> &tab, int ntab, int M, int Kd, bool mixed) {
    g.M = M;
    g.Kd = Kd;
    g.ntab = ntab;
    g.Kpad = (Kd + 31) / 32 * 32;
    g.Mpad = (M + 15) / 16 * 16;
    g.tab = dev_upload(tab);
    if (!mixed) return;
    std::vector<uint16_t> sl((size_t)ntab * kSlicesS * g.Mpad * g.Kpad, 0);
    std::vector<int32_t> ex((size_t)ntab * g.Mpad, 0);
    for (int t = 0; t < ntab; ++t)
        for (int i = 0; i < M; ++i) {
            const double *row = &tab[((size_t)t * M + i) * Kd];
            double m = 0.0;
            for (int k = 0; k < Kd; ++k) m = std::max(m, std::fabs(row[k]));
            int e = slice_expo(m);
            ex[(size_t)t * g.Mpad + i] = e;
            for (int k = 0; k < Kd; ++k) {
                double y = std::ldexp(row[k], -e);
                for (int s = 0; s < kSlicesS; ++s) {
                    y = std::ldexp(y, kSliceBitsB);
                    double q = std::rint(y);
                    y -= q;
                    sl[(((size_t)t * kSlicesS + s) * g.Mpad + i) * g.Kpad + k] = bf16_bits_exact(q);
                }
            }
        }
    g.tslices = dev_upload(sl);
    g.texpo = dev_upload(ex);
}

// Opt the sliced engine into its dynamic shared memory (once per device, at setup).
void gemm_prepare_device() {
    const size_t smem = 2 * X_STAGE * sizeof(uint16_t);
    VPX_CUDA(cudaFuncSetAttribute(k_gemm_sliced<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VPX_CUDA(cudaFuncSetAttribute(k_gemm_sliced<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}

void gemm_pass_free(GemmPass &g) {
    dev_free(g.tab);
    dev_free(g.tslices);
    dev_free(g.texpo);
    dev_free(g.pairs);
    dev_free(g.tiles);
    g.n_pairs = g.n_tiles = 0;
}

void gemm_tc_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, int *status, void *s);

void gemm_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, bool mixed, void *sv) {
    if (g.n_tiles == 0) return;
    cudaStream_t s = (cudaStream_t)sv;
    const bool no_tc = getenv("VPX_NO_TC") != nullptr;
    if (mixed && !no_tc && gemm_tc_eligible(g)) {
        gemm_tc_run(g, vs, out, ldo, nrhs, g.status, sv);
        return;
    }
    if (!mixed) {
        dim3 grid(g.n_tiles, (g.M + G_M - 1) / G_M, nrhs);
        k_gemm_fp64<<<grid, 256, 0, s>>>(g.M, g.Kd, g.tab, g.tiles, g.pairs, vs.base, vs.ld, vs.stride, out, ldo, g.add);
        VPX_LAUNCH("k_gemm_fp64");
        return;
    }
    SlicedArgs a;
    a.M = g.M;
    a.Mpad = g.Mpad;
    a.Kpad = g.Kpad;
    a.nvec = vs.nvec;
    a.tslices = g.tslices;
    a.texpo = g.texpo;
    a.tiles = g.tiles;
    a.pairs = g.pairs;
    a.vslices = vs.slices;
    a.vexpo = vs.expo;
    a.out = out;
    a.ldo = ldo;
    a.add = g.add;
    const size_t smem = 2 * X_STAGE * sizeof(uint16_t);
    dim3 grid(g.n_tiles, (g.M + X_M - 1) / X_M, nrhs);
    if (g.slices >= 6) k_gemm_sliced<6><<<grid, 256, smem, s>>>(a);
    else k_gemm_sliced<5><<<grid, 256, smem, s>>>(a);
    VPX_LAUNCH("k_gemm_sliced");
}

void slice_vectors(const VecSet &vs, int first, int count, int Kd, int Kpad, int nrhs, void *sv) {
    if (count <= 0) return;
    k_slice_vec<<<dim3(count, nrhs), 128, 0, (cudaStream_t)sv>>>(vs.base, vs.ld, vs.stride, first, Kd, Kpad, vs.nvec,
                                                                 vs.slices, vs.expo);
    VPX_LAUNCH("k_slice_vec");
}

}  // namespace vpx
