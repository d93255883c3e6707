// gemm_frag.cu -- the exact-slice table GEMM (gemm.cuh) for the passes whose
// work per launch is small: every far-field translation (L2M, M2M, M2L, S2L,
// L2L, L2T, M2T).  These run level by level on the critical path, so the
// kernel is built for latency rather than peak rate:
//
//  * the table operand never touches shared memory: its bf16 slices are stored
//    in mma.sync m16n8k16 A-fragment order (one 16-byte load per lane per slice
//    and 16-deep k step, coalesced across the warp, L2-resident);
//  * a CTA covers all rows of one row block (one warp per 16 rows) for 32
//    pairs; the inner dimension is split across CTAs in 64-deep chunks where it
//    is long (leaf values, Kd = K^2), results meeting in the output atomics;
//  * source vectors with Kd <= 128 (expansions) are sliced by the CTA itself
//    as it stages them (no separate slicing launch); leaf values arrive
//    pre-sliced and are copied with cp.async.
//
// Slice products a_k b_l with k + l <= S + 1 accumulate per order d = k + l in
// fp32, exactly (order sums stay below 2^24 for the 64-deep chunks of
// pre-sliced vectors and for the inner dimensions <= 128 of on-the-fly sliced
// ones, slice_math.cuh), and the slice_math.cuh epilogue combines them.
#include <cuda_bf16.h>

#include <algorithm>

#include "bulk.cuh"
#include "dev_common.cuh"
#include "gemm.cuh"
#include "slice_math.cuh"

namespace vpx {

constexpr int F_KC_PRE = 4;        // k16 blocks per CTA chunk for pre-sliced vectors
constexpr int F_MAX_KB_FLY = 16;   // on-the-fly slicing: Kpad <= 256 (32 pairs x 256 doubles staged: 166 KB)
constexpr int F_MAX_KB_WHOLE = 8;  // pre-sliced vectors up to this many k16 blocks are staged whole
constexpr int F_MAX_WARPS = 6;     // m16 blocks (warps) per CTA: 96 rows, two CTAs per SM

struct FragArgs {
    int M, Mpad, Kd, Kpad, MB, KB;
    int wm, rb, kc, ks;            // warps (m16 blocks) per CTA, row blocks, k16 blocks per chunk, chunks
    const uint4 *tfrag;            // [ntab][kSlicesS][MB][KB][32]
    const int32_t *texpo;          // [ntab][Mpad]
    const GTile *tiles;            // 8 NT pairs each
    const GPair *pairs;
    const double *vbase;           // vectors (on-the-fly slicing)
    int64_t vld;
    int vstride;
    const uint16_t *vslices;       // or pre-sliced: [rhs][nvec][kSlicesS][vkpad]
    const int32_t *vexpo;          // [rhs][nvec]
    int nvec, vkpad;
    double *out;
    int64_t ldo;
    int add;
    int bulk;                      // on-the-fly vectors may be staged by TMA bulk copies (16-byte aligned)
    int *status;
};

__device__ inline void frag_cp16(void *smem, const void *gmem, int bytes) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes));
}

__device__ inline void frag_mma(float (&c)[4], const uint4 &a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// grid: x = tile x row block x k chunk, y = rhs; block = wm warps; NT n8 tiles
// (8 NT pairs) per CTA
template <int S, bool FLY, int NT>
__global__ void __launch_bounds__(192, 2) k_gemm_frag(FragArgs a) {
    pdl_entry();
    constexpr int NP = 8 * NT;
    extern __shared__ __align__(16) uint16_t bs[];   // [S][NP][ldb] slices, then (FLY) [NP][Kd] doubles
    __shared__ GPair s_pr[NP];
    __shared__ int s_ve[NP];
    __shared__ SliceScale s_ps[NP];
    __shared__ __align__(8) uint64_t s_bar;
    const int per_tile = a.rb * a.ks;
    const int ti = blockIdx.x / per_tile, rem = blockIdx.x % per_tile;
    const int rbi = rem / a.ks, ksi = rem % a.ks;
    const int rhs = blockIdx.y;
    const GTile tile = a.tiles[ti];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int ldb = a.kc * 16 + 8;
    const int kb0 = ksi * a.kc;
    const int nkb = min(a.kc, a.KB - kb0);
    const int mb = rbi * a.wm + warp;
    // the first table fragments do not depend on the vectors: request them now
    const size_t sstride = (size_t)a.MB * a.KB * 32;
    const uint4 *Af = a.tfrag + (((size_t)tile.tab * kSlicesS * a.MB + min(mb, a.MB - 1)) * a.KB + kb0) * 32 + lane;
    uint4 af[S];
#pragma unroll
    for (int s = 0; s < S; ++s) af[s] = __ldg(Af + s * sstride);
    // the rows' exponents do not depend on the vectors either
    int row_e[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int i = mb * 16 + (lane >> 2) + rr * 8;
        row_e[rr] = (mb < a.MB && i < a.M) ? a.texpo[(size_t)tile.tab * a.Mpad + i] : 0;
    }
    for (int n = threadIdx.x; n < NP; n += blockDim.x)
        s_pr[n] = (n < tile.count) ? a.pairs[tile.first + n] : GPair{0, 0, -1, 0.0};
    if (FLY && threadIdx.x == 0) bulk_bar_init(&s_bar);
    __syncthreads();

    // ---- stage the source vectors' slices for k in [16 kb0, 16 (kb0 + nkb))
    if (FLY) {
        // the NP vectors arrive at once (TMA bulk copies when aligned), then one
        // warp per vector takes its exponent and slices from shared memory
        double *xs = reinterpret_cast<double *>(bs + (size_t)S * NP * ldb);
        bool ok = true;
        if (a.bulk) {
            if (threadIdx.x == 0) {
                const uint32_t bytes = (uint32_t)(a.Kd * sizeof(double));
                bulk_expect(&s_bar, bytes * tile.count);
                for (int n = 0; n < tile.count; ++n)
                    bulk_copy(xs + (size_t)n * a.Kd, a.vbase + rhs * a.vld + (int64_t)s_pr[n].src * a.vstride, bytes,
                              &s_bar);
            }
            ok = __syncthreads_and(bulk_wait(&s_bar, 0));
        } else {
            for (int c = threadIdx.x; c < tile.count * a.Kd; c += blockDim.x) {
                const int n = c / a.Kd, j = c % a.Kd;
                xs[c] = a.vbase[rhs * a.vld + (int64_t)s_pr[n].src * a.vstride + j];
            }
            __syncthreads();
        }
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.status, VPX_ERR_TIMEOUT);
            return;
        }
        for (int n = warp; n < NP; n += nwarp) {
            const bool live = n < tile.count;
            const double *x = xs + (size_t)n * a.Kd;
            uint64_t m = 0;
            if (live)
                for (int j = lane; j < a.Kd; j += 32) {
                    const uint64_t t = slice_abs_bits(x[j]);
                    m = t > m ? t : m;
                }
            const int e = slice_warp_expo(m);
            for (int j = lane; j < nkb * 16; j += 32) {
                const int k = kb0 * 16 + j;
                uint16_t d[kSlicesS];
                slice_digits((live && k < a.Kd) ? slice_fixed_point(x[k], e) : 0, d);
#pragma unroll
                for (int s = 0; s < S; ++s) bs[(s * NP + n) * ldb + j] = d[s];
            }
            if (lane == 0) s_ve[n] = e;
        }
    } else {
        const int cpr = nkb * 2;   // 16-byte chunks per (slice, vector) row
        for (int c = threadIdx.x; c < S * NP * cpr; c += blockDim.x) {
            const int s = c / (NP * cpr), r = c % (NP * cpr), n = r / cpr, q = r % cpr;
            const bool ok = n < tile.count;
            const uint16_t *src =
                a.vslices + (((size_t)rhs * a.nvec + (ok ? s_pr[n].src : 0)) * kSlicesS + s) * a.vkpad + kb0 * 16 + q * 8;
            frag_cp16(bs + (s * NP + n) * ldb + q * 8, src, ok ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        for (int n = threadIdx.x; n < NP; n += blockDim.x)
            s_ve[n] = (n < tile.count) ? a.vexpo[(size_t)rhs * a.nvec + s_pr[n].src] : 0;
        asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncthreads();
    for (int n = threadIdx.x; n < NP; n += blockDim.x)
        s_ps[n] = slice_pair_scale(s_pr[n].scale, s_ve[n] - 2 * kSliceBitsB);
    __syncthreads();

    // ---- warp w: rows of m16 block rbi * wm + w, all NP pairs
    if (mb >= a.MB) return;
    const int g = lane >> 2, tq = lane & 3;
    float acc[S][NT][4];
#pragma unroll
    for (int d = 0; d < S; ++d)
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[d][t][r] = 0.f;
    for (int kb = 0; kb < nkb; ++kb) {
        uint4 an[S];
        if (kb + 1 < nkb) {
#pragma unroll
            for (int s = 0; s < S; ++s) an[s] = __ldg(Af + s * sstride + (kb + 1) * 32);
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const uint16_t *Br = bs + (l * NP + t * 8 + g) * ldb + kb * 16 + tq * 2;
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(Br);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(Br + 8);
#pragma unroll
                for (int s = 0; s + l < S; ++s) frag_mma(acc[s + l][t], af[s], b0, b1);
            }
        }
        if (kb + 1 < nkb) {
#pragma unroll
            for (int s = 0; s < S; ++s) af[s] = an[s];
        }
    }

    // ---- epilogue
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int i = mb * 16 + g + rr * 8;
        if (i >= a.M) continue;
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int n = t * 8 + tq * 2 + half;
                const int64_t dst = s_pr[n].dst;
                if (dst < 0) continue;
                float acc_d[S];
#pragma unroll
                for (int d = 0; d < S; ++d) acc_d[d] = acc[d][t][rr * 2 + half];
                const double val = slice_output<S>(acc_d, s_ps[n], row_e[rr]);
                double *o = a.out + rhs * a.ldo + dst + i;
                if (a.add) atomicAdd(o, val);
                else *o = val;
            }
    }
}

// ------------------------------------------------------------------ host

static size_t frag_smem(int S, int np, int kc, bool fly, int Kd) {
    size_t b = (size_t)S * np * (kc * 16 + 8) * sizeof(uint16_t);
    return fly ? b + (size_t)np * Kd * sizeof(double) : b;
}

template <int S, bool FLY, int NT>
static void frag_attr() {
    const int smax = (int)frag_smem(kSlicesS, 32, F_MAX_KB_FLY, true, 16 * F_MAX_KB_FLY);
    VPX_CUDA(cudaFuncSetAttribute(k_gemm_frag<S, FLY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
}

void gemm_frag_prepare_device() {
    frag_attr<kSlicesS, true, 1>();
    frag_attr<kSlicesS, true, 4>();
    frag_attr<kSlicesS, false, 1>();
    frag_attr<kSlicesS, false, 4>();
}

bool gemm_frag_eligible(const GemmPass &g, const VecSet &vs) {
    if (!g.tfrag || g.Kpad > 512) return false;
    return vs.slices != nullptr || g.Kpad <= 16 * F_MAX_KB_FLY;
}

template <int S, bool FLY>
static void frag_launch(int np, dim3 grid, int threads, size_t smem, cudaStream_t st, const FragArgs &a) {
    if (np == 8) launch_pdl(k_gemm_frag<S, FLY, 1>, grid, dim3(threads), smem, st, a);
    else launch_pdl(k_gemm_frag<S, FLY, 4>, grid, dim3(threads), smem, st, a);
}

void gemm_frag_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s) {
    if (g.n_tiles_f == 0) return;
    FragArgs a;
    a.M = g.M;
    a.Mpad = g.Mpad;
    a.Kd = g.Kd;
    a.Kpad = g.Kpad;
    a.MB = g.Mpad / 16;
    a.KB = g.Kpad / 16;
    a.wm = std::min(F_MAX_WARPS, a.MB);
    a.rb = (a.MB + a.wm - 1) / a.wm;
    const bool fly = vs.slices == nullptr;
    a.kc = (fly || a.KB <= F_MAX_KB_WHOLE) ? a.KB : F_KC_PRE;
    a.ks = (a.KB + a.kc - 1) / a.kc;
    a.tfrag = reinterpret_cast<const uint4 *>(g.tfrag);
    a.texpo = g.texpo;
    a.tiles = g.tiles_f;
    a.pairs = g.pairs;
    a.vbase = vs.base;
    a.vld = vs.ld;
    a.vstride = vs.stride;
    a.vslices = vs.slices;
    a.vexpo = vs.expo;
    a.nvec = vs.nvec;
    a.vkpad = vs.kpad;
    a.out = out;
    a.ldo = ldo;
    a.add = g.add;
    a.status = g.status;
    a.bulk = fly && (a.Kd % 2 == 0) && (vs.stride % 2 == 0) && (vs.ld % 2 == 0) &&
             (reinterpret_cast<uintptr_t>(vs.base) % 16 == 0);
    if (a.ks > 1 && !a.add) fail(VPX_ERR_ARG, "a pass split along its inner dimension must accumulate");
    if (!fly && vs.kpad < g.Kpad) fail(VPX_ERR_ARG, "pre-sliced vectors shorter than the table's inner dimension");
    const size_t smem = frag_smem(kSlicesS, g.np_f, a.kc, fly, a.Kd);
    dim3 grid((unsigned)(g.n_tiles_f * a.rb * a.ks), (unsigned)nrhs);
    cudaStream_t st = (cudaStream_t)s;
    if (fly) frag_launch<kSlicesS, true>(g.np_f, grid, a.wm * 32, smem, st, a);
    else frag_launch<kSlicesS, false>(g.np_f, grid, a.wm * 32, smem, st, a);
    VPX_LAUNCH("k_gemm_frag");
}

}  // namespace vpx
