// gemm_tc.cu -- the exact bf16-slice table GEMM (gemm.cuh) on the 5th-generation
// tensor cores: tcgen05.mma with operands in shared memory and the fp32
// accumulators in tensor memory.
//
// Tile: 128 table rows x 64 pairs per CTA (256 threads).  Per 32-deep k stage
// the S table slices (128 x 32 each) and the S vector slices (64 x 32 each)
// are copied with cp.async into the no-swizzle K-major canonical layout
// (8-row x 16-byte core matrices; K-adjacent core matrices LBO bytes apart,
// row groups 128 bytes apart).  One thread issues, per 16-deep k step, the
// S(S+1)/2 slice products a_k b_l with k + l <= S + 1 into the accumulator of
// order d = k + l (M = 128, N = 64, K = 16 each; 5 orders x 64 columns of
// TMEM), then tcgen05.commit arrives on the stage's mbarrier.  Three stage
// buffers: a buffer is refilled only after the mbarrier of the products that
// read it has flipped.  Each order sum is exact in fp32 (see gemm.cu); the
// epilogue reads the accumulators with tcgen05.ld and recombines them exactly
// as the mma.sync engine does.  Every mbarrier wait is bounded: on timeout the
// CTA sets VPX_ERR_TIMEOUT, releases its tensor memory and returns.
#include <cuda_bf16.h>

#include "dev_common.cuh"
#include "gemm.cuh"
#include "slice_math.cuh"

namespace vpx {

constexpr int TC_M = 128, TC_N = 64, TC_K = 32, TC_STAGES = 3, TC_S = 5;
constexpr int TC_A_SLICE = TC_M * TC_K;                     // bf16 per A slice tile
constexpr int TC_B_SLICE = TC_N * TC_K;                     // bf16 per B slice tile
constexpr int TC_STAGE = TC_S * (TC_A_SLICE + TC_B_SLICE);  // bf16 per stage
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr long long TC_SPIN_LIMIT = 1ll << 26;

// instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major canonical layout
__device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // fixed 0b001 in bits 46-48
    return d;                 // base offset 0, swizzle mode 0 (none)
}

__device__ inline void tc_cp16(uint32_t saddr, const void *g, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(bytes));
}

__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

struct TcArgs {
    int M, Mpad, Kpad, nvec;
    const uint16_t *tslices;   // [ntab][6][Mpad][Kpad]
    const int32_t *texpo;
    const GTile *tiles;
    const GPair *pairs;
    const uint16_t *vslices;   // [rhs][nvec][6][Kpad]
    const int32_t *vexpo;
    double *out;
    int64_t ldo;
    int add;
    int *status;
};

__global__ void __launch_bounds__(256, 1) k_gemm_tc(TcArgs a) {
    extern __shared__ __align__(1024) uint16_t tsm[];
    __shared__ __align__(8) uint64_t s_bar[TC_STAGES];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ SliceScale s_ps[TC_N];
    __shared__ int64_t s_pdst[TC_N];
    __shared__ int s_src[TC_N];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GTile tile = a.tiles[blockIdx.x];
    const int m0 = blockIdx.y * TC_M, rhs = blockIdx.z;
    const uint16_t *T = a.tslices + (size_t)tile.tab * kSlicesS * a.Mpad * a.Kpad;
    const uint16_t *VS = a.vslices + (size_t)rhs * a.nvec * kSlicesS * a.Kpad;

    if (tid < TC_N) s_src[tid] = (tid < tile.count) ? a.pairs[tile.first + tid].src : 0;
    if (tid == 0) {
        s_fail = 0;
        for (int i = 0; i < TC_STAGES; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_bar[i])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t base = smem_u32(tsm);

    // k stage kt -> buffer kt % 3: A slice s at s * 8 KB, B slice l after the A slices
    auto stage_fill = [&](int buf, int k0) {
        const uint32_t sb = base + (uint32_t)(buf * TC_STAGE * 2);
        for (int c = tid; c < TC_S * TC_M * 4; c += 256) {
            int s = c / (TC_M * 4), rem = c % (TC_M * 4), r = rem >> 2, q = rem & 3;
            int gr = m0 + r;
            const uint16_t *src = T + ((size_t)s * a.Mpad + (gr < a.Mpad ? gr : 0)) * a.Kpad + k0 + q * 8;
            uint32_t dst = sb + (uint32_t)(s * TC_A_SLICE * 2 + q * (TC_M * 16) + (r >> 3) * 128 + (r & 7) * 16);
            tc_cp16(dst, src, gr < a.Mpad ? 16 : 0);
        }
        for (int c = tid; c < TC_S * TC_N * 4; c += 256) {
            int s = c / (TC_N * 4), rem = c % (TC_N * 4), n = rem >> 2, q = rem & 3;
            bool ok = n < tile.count;
            const uint16_t *src = VS + ((size_t)s_src[n] * kSlicesS + s) * a.Kpad + k0 + q * 8;
            uint32_t dst = sb + (uint32_t)(TC_S * TC_A_SLICE * 2 + s * TC_B_SLICE * 2 + q * (TC_N * 16) +
                                           (n >> 3) * 128 + (n & 7) * 16);
            tc_cp16(dst, src, ok ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    const int nk = a.Kpad / TC_K;
    uint32_t phase[TC_STAGES] = {0, 0, 0};
    int committed[TC_STAGES] = {0, 0, 0};
    bool first_d[TC_S] = {true, true, true, true, true};
    bool ok = true;
    stage_fill(0, 0);
    if (nk > 1) stage_fill(1, TC_K);
    for (int kt = 0; kt < nk && ok; ++kt) {
        const int buf = kt % TC_STAGES;
        if (kt + 2 < nk) {
            const int nb = (kt + 2) % TC_STAGES;
            if (committed[nb]) {   // products of stage kt-1 read this buffer
                if (!mbar_wait(smem_u32(&s_bar[nb]), phase[nb])) ok = false;
                phase[nb] ^= 1u;
                committed[nb] = 0;
            }
            stage_fill(nb, (kt + 2) * TC_K);
            asm volatile("cp.async.wait_group 2;\n" ::);
        } else if (kt + 1 < nk) {
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (!ok) {
            if (tid == 0) atomicExch(&s_fail, 1);
        }
        __syncthreads();
        if (s_fail) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sb = base + (uint32_t)(buf * TC_STAGE * 2);
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk) {
#pragma unroll
                for (int l = 0; l < TC_S; ++l) {
                    const uint32_t baddr = sb + (uint32_t)(TC_S * TC_A_SLICE * 2 + l * TC_B_SLICE * 2 + kk * 2 * (TC_N * 16));
                    const uint64_t bdesc = smem_desc(baddr, TC_N * 16, 128);
#pragma unroll
                    for (int s = 0; s < TC_S; ++s) {
                        if (s + l >= TC_S) continue;
                        const uint32_t aaddr = sb + (uint32_t)(s * TC_A_SLICE * 2 + kk * 2 * (TC_M * 16));
                        const uint64_t adesc = smem_desc(aaddr, TC_M * 16, 128);
                        const int d = s + l;
                        const uint32_t dt = tmem + (uint32_t)(d * TC_N);
                        const uint32_t acc = first_d[d] ? 0u : 1u;
                        first_d[d] = false;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
                            "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(acc));
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&s_bar[buf]))
                         : "memory");
        }
        committed[buf] = 1;
    }
    // wait for the last products of every buffer
    if (ok) {
        for (int b = 0; b < TC_STAGES; ++b)
            if (committed[b]) {
                if (!mbar_wait(smem_u32(&s_bar[b]), phase[b])) ok = false;
                phase[b] ^= 1u;
                committed[b] = 0;
            }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    if (!ok) atomicExch(&s_fail, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!s_fail) {
        // epilogue: per-pair scales once per CTA; warp w reads TMEM lanes 32 (w % 4)..
        // (one table row per thread) for the pair columns of half w / 4
        if (tid < TC_N) {
            s_pdst[tid] = -1;
            s_ps[tid] = SliceScale{0.f, 0.f, 0};
            if (tid < tile.count) {
                const GPair pr = a.pairs[tile.first + tid];
                s_ps[tid] = slice_pair_scale(pr.scale, a.vexpo[(size_t)rhs * a.nvec + pr.src] - 2 * kSliceBitsB);
                s_pdst[tid] = rhs * a.ldo + pr.dst;
            }
        }
        __syncthreads();
        const int q4 = warp & 3, half = warp >> 2;
        const int i = m0 + q4 * 32 + lane;
        const int row_e = (i < a.M) ? a.texpo[(size_t)tile.tab * a.Mpad + i] : 0;
        for (int c0 = half * (TC_N / 2); c0 < (half + 1) * (TC_N / 2); c0 += 16) {
            uint32_t r[TC_S][16];
#pragma unroll
            for (int d = 0; d < TC_S; ++d) {
                const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(d * TC_N + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                    : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3]), "=r"(r[d][4]), "=r"(r[d][5]),
                      "=r"(r[d][6]), "=r"(r[d][7]), "=r"(r[d][8]), "=r"(r[d][9]), "=r"(r[d][10]), "=r"(r[d][11]),
                      "=r"(r[d][12]), "=r"(r[d][13]), "=r"(r[d][14]), "=r"(r[d][15])
                    : "r"(ta));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (i < a.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = c0 + j;
                    if (s_pdst[n] < 0) continue;
                    float acc[TC_S], hi, lo;
#pragma unroll
                    for (int d = 0; d < TC_S; ++d) acc[d] = __uint_as_float(r[d][j]);
                    slice_recombine<TC_S>(acc, hi, lo);
                    const double val = slice_output(hi, lo, s_ps[n], row_e);
                    double *o = a.out + s_pdst[n] + i;
                    if (a.add) atomicAdd(o, val);
                    else *o = val;
                }
            }
        }
    } else if (tid == 0) {
        set_status(a.status, VPX_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

// ------------------------------------------------------------------ host

size_t gemm_tc_smem() { return (size_t)TC_STAGES * TC_STAGE * sizeof(uint16_t); }

void gemm_tc_prepare_device() {
    VPX_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem()));
}

bool gemm_tc_eligible(const GemmPass &g) { return g.slices == TC_S && g.Mpad % TC_M == 0 && g.Kpad % TC_K == 0; }

void gemm_tc_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, int *status, void *s) {
    if (g.n_tiles == 0) return;
    TcArgs a;
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
    a.status = status;
    dim3 grid(g.n_tiles, g.Mpad / TC_M, nrhs);
    k_gemm_tc<<<grid, 256, gemm_tc_smem(), (cudaStream_t)s>>>(a);
    VPX_LAUNCH("k_gemm_tc");
}

}  // namespace vpx
