// gemm_ws.cu -- the exact-slice table GEMM (gemm.cuh) on the 5th-generation
// tensor cores as a warp-specialised pipeline.
//
// One CTA computes, for one table and one block of its rows and one block of
// its pairs, the S(S+1)/2 slice products a_k b_l (0-based, k + l <= S - 1)
// into S fp32 accumulators in tensor memory (one per order d = k + l; exact,
// see slice_math.cuh), then recombines them.  Two orientations:
//
//   TM = true  (instantiated): M = 128 table rows, N = 48 pairs, S = 5 (five
//              orders of 48 columns in a 256-column tensor-memory
//              allocation, and three stages in 82.5 KB of shared memory, so
//              that two CTAs share an SM and each hides the other's set-up,
//              pipeline fill and epilogue): the near field, L2M and lists i+
//              and i-;
//   TM = false: M = 128 pairs, N = table rows (the template allows it; no
//              pass is routed to it).
//
// Roles (256 threads):
//   warp 0, one lane   table tiles by TMA bulk copies (cp.async.bulk): the
//                      table slices are stored with 8-column chunks
//                      interleaved ([tab][slice][Kpad/8][Mpad][8]), so the rows
//                      x 16 bytes of one chunk are contiguous and land as the
//                      no-swizzle K-major core-matrix layout in one copy;
//   warp 1, one lane   issues tcgen05.mma for a stage once its full barrier
//                      flips, then tcgen05.commit to the stage's empty barrier
//                      (and to the done barrier after the last stage);
//   warps 2..7         gather the pairs' vector slices with 16-byte cp.async
//                      into the same layout; cp.async.mbarrier.arrive.noinc
//                      makes each thread's copies one arrival on the full
//                      barrier;
//   all warps          the epilogue once the done barrier flips.
// Stages form a ring of TW_STAGES buffers of TW_K = 16 inner indices each.  Every
// barrier wait is bounded; a timeout sets VPX_ERR_TIMEOUT, skips the epilogue,
// and the CTA still releases its tensor memory.
#include <cuda_bf16.h>

#include <cstdlib>

#include "bulk.cuh"
#include "dev_common.cuh"
#include "gemm.cuh"
#include "slice_math.cuh"

namespace vpx {

constexpr int TW_M = 128, TW_K = 16, TW_STAGES = 3, TW_THREADS = 256, TW_PROD0 = 64;   // producers: threads 64..255
constexpr int TW_NPROD = TW_THREADS - TW_PROD0;
constexpr int TW_KQ = TW_K / 8;   // 8-column chunks per stage

// tensor-memory columns to allocate: a power of two >= 32
constexpr uint32_t tw_tmem_cols(int n) { return n <= 32 ? 32u : 2u * tw_tmem_cols((n + 1) / 2); }

__device__ inline uint32_t tw_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t tw_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // fixed 0b001 in bits 46-48; base offset 0, no swizzle
    return d;
}

__device__ inline bool tw_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait_bounded(tw_smem(bar), parity, kWaitLimitNs, 0);
}

struct WsArgs {
    int M, Mpad, Kpad, nvec;
    const uint16_t *tint;      // [ntab][S][Kpad/8][Mpad][8] table slices, column chunks interleaved
    const int32_t *texpo;      // [ntab][Mpad]
    const GTile *tiles;
    const GPair *pairs;
    const uint16_t *vslices;   // [rhs][nvec][S][Kpad]
    const int32_t *vexpo;
    double *out;
    int64_t ldo;
    int add;
    int *status;
};

template <bool TM, int S, int NB>
struct WsShape {
    static constexpr int TR = TM ? TW_M : NB;     // table rows per CTA
    static constexpr int VR = TM ? NB : TW_M;     // pairs per CTA
    static constexpr int A_SLICE = TW_M * TW_K;   // bf16 per A slice
    static constexpr int B_SLICE = NB * TW_K;     // bf16 per B slice
    static constexpr int STAGE = S * (A_SLICE + B_SLICE);
    static constexpr uint32_t T_BYTES = (uint32_t)(S * TW_KQ * TR * 16);   // table bytes per stage
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NB >> 3) << 17) |
                                      ((uint32_t)(TW_M >> 4) << 24);
    static constexpr size_t SMEM = (size_t)TW_STAGES * STAGE * sizeof(uint16_t);
    static constexpr uint32_t TMEM_COLS = tw_tmem_cols(S * NB);
    static_assert(TMEM_COLS <= 512, "accumulators exceed tensor memory");
};

// grid: x = tile of pairs, y = block of table rows, z = rhs
template <bool TM, int S, int NB>
__global__ void __launch_bounds__(TW_THREADS, 2) k_gemm_ws(WsArgs a) {
    pdl_entry();
    typedef WsShape<TM, S, NB> Sh;
    extern __shared__ __align__(1024) uint16_t wsm[];
    __shared__ __align__(8) uint64_t full[TW_STAGES], empty[TW_STAGES], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ int s_src[Sh::VR];
    __shared__ SliceScale s_ps[Sh::VR];
    __shared__ int64_t s_pdst[Sh::VR];
    __shared__ int s_rowe[Sh::TR];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GTile tile = a.tiles[blockIdx.x];
    const int row0 = blockIdx.y * Sh::TR, rhs = blockIdx.z;
    const int nk = a.Kpad / TW_K;

    for (int i = tid; i < Sh::VR; i += TW_THREADS) {
        s_src[i] = 0;
        s_pdst[i] = -1;
        s_ps[i] = SliceScale{1.0, 0, 1};
        if (i < tile.count) {
            const GPair pr = a.pairs[tile.first + i];
            s_src[i] = pr.src;
            s_pdst[i] = rhs * a.ldo + pr.dst;
            s_ps[i] = slice_pair_scale(pr.scale, a.vexpo[(size_t)rhs * a.nvec + pr.src] - 2 * kSliceBitsB);
        }
    }
    for (int i = tid; i < Sh::TR; i += TW_THREADS)
        s_rowe[i] = (row0 + i < a.M) ? a.texpo[(size_t)tile.tab * a.Mpad + row0 + i] : 0;
    if (tid == 0) {
        // TMA destinations must be 128-byte aligned: refuse to start otherwise
        s_fail = (tw_smem(wsm) & 127u) != 0u;
        for (int i = 0; i < TW_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tw_smem(&full[i])), "r"(1 + TW_NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tw_smem(&empty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tw_smem(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tw_smem(&s_tmem)),
                     "r"(Sh::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t base = tw_smem(wsm);
    const uint32_t t_off = TM ? 0u : (uint32_t)(S * Sh::A_SLICE * 2);   // table operand within a stage
    const uint32_t v_off = TM ? (uint32_t)(S * Sh::A_SLICE * 2) : 0u;   // vector operand within a stage
    const uint32_t t_lbo = (uint32_t)(Sh::TR * 16), v_lbo = (uint32_t)(Sh::VR * 16);
    const uint32_t t_slice = (uint32_t)(Sh::TR * TW_K * 2), v_slice = (uint32_t)(Sh::VR * TW_K * 2);

    if (warp == 0) {
        // ---- table producer: one bulk copy per (slice, 8-column chunk): TR rows x 16 bytes,
        // contiguous in the interleaved layout and in the core-matrix layout alike
        if (lane == 0 && !s_fail) {
            const int kc_n = a.Kpad / 8;
            for (int kt = 0; kt < nk; ++kt) {
                const int b = kt % TW_STAGES;
                if (kt >= TW_STAGES && !tw_wait(&empty[b], ((kt / TW_STAGES) - 1) & 1)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tw_smem(&full[b])),
                             "r"(Sh::T_BYTES)
                             : "memory");
                const uint32_t sb = base + (uint32_t)(b * Sh::STAGE * 2) + t_off;
                for (int s2 = 0; s2 < S; ++s2)
                    for (int q = 0; q < TW_KQ; ++q) {
                        const size_t chunk = ((size_t)(tile.tab * kSlicesS + s2) * kc_n + kt * TW_KQ + q) * a.Mpad + row0;
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                                sb + s2 * t_slice + q * t_lbo),
                            "l"(a.tint + chunk * 8), "r"((uint32_t)(Sh::TR * 16)), "r"(tw_smem(&full[b]))
                            : "memory");
                    }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            for (int kt = 0; kt < nk; ++kt) {
                const int b = kt % TW_STAGES;
                if (s_fail || !tw_wait(&full[b], (kt / TW_STAGES) & 1)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // cp.async writes -> async proxy
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                // descriptors of this stage's slice 0, k step 0; the rest by adding (offset >> 4)
                const uint32_t sb = base + (uint32_t)(b * Sh::STAGE * 2);
                const uint64_t t0 = tw_desc(sb + t_off, t_lbo, 128), v0 = tw_desc(sb + v_off, v_lbo, 128);
                const uint64_t a0 = TM ? t0 : v0, b0 = TM ? v0 : t0;
                constexpr uint32_t a_slice16 = (uint32_t)(TW_M * TW_K * 2) >> 4, b_slice16 = (uint32_t)(NB * TW_K * 2) >> 4;
                constexpr uint32_t a_kk16 = (uint32_t)(2 * TW_M * 16) >> 4, b_kk16 = (uint32_t)(2 * NB * 16) >> 4;
#pragma unroll
                for (int kk = 0; kk < TW_K / 16; ++kk) {
#pragma unroll
                    for (int l = 0; l < S; ++l) {
                        const uint64_t bdesc = b0 + (uint64_t)(l * b_slice16 + kk * b_kk16);
#pragma unroll
                        for (int s2 = 0; s2 < S; ++s2) {
                            if (s2 + l >= S) continue;
                            const uint64_t adesc = a0 + (uint64_t)(s2 * a_slice16 + kk * a_kk16);
                            const uint32_t dt = tmem + (uint32_t)((s2 + l) * NB);
                            // l = 0 meets every order d = s2 first: those products overwrite
                            const uint32_t acc = (kt == 0 && kk == 0 && l == 0) ? 0u : 1u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
                                "l"(adesc), "l"(bdesc), "r"(Sh::IDESC), "r"(acc));
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 tw_smem(&empty[b]))
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             tw_smem(&done))
                         : "memory");
        }
    } else {
        // ---- vector producers: 16-byte chunks of the pairs' slices; a thread's
        // chunks are the same (slice, pair, column chunk) at every stage
        constexpr int NCH = (S * Sh::VR * TW_KQ + TW_NPROD - 1) / TW_NPROD;
        const int pt = tid - TW_PROD0;
        const uint16_t *VS = a.vslices + (size_t)rhs * a.nvec * kSlicesS * a.Kpad;
        const uint16_t *srcp[NCH];
        uint32_t dsto[NCH];
        int nbytes[NCH];
#pragma unroll
        for (int i = 0; i < NCH; ++i) {
            const int c = pt + i * TW_NPROD;
            const int s2 = c / (Sh::VR * TW_KQ), rem = c % (Sh::VR * TW_KQ), r = rem / TW_KQ, q = rem % TW_KQ;
            const bool live = c < S * Sh::VR * TW_KQ;
            nbytes[i] = (live && r < tile.count) ? 16 : 0;
            srcp[i] = VS + ((size_t)(live ? s_src[r] : 0) * kSlicesS + (live ? s2 : 0)) * a.Kpad + q * 8;
            dsto[i] = live ? (uint32_t)(s2 * v_slice + q * v_lbo + (r >> 3) * 128 + (r & 7) * 16) : 0u;
        }
        for (int kt = 0; kt < nk; ++kt) {
            const int b = kt % TW_STAGES;
            if (kt >= TW_STAGES && !tw_wait(&empty[b], ((kt / TW_STAGES) - 1) & 1)) {
                atomicExch(&s_fail, 1);
                break;
            }
            const uint32_t sb = base + (uint32_t)(b * Sh::STAGE * 2) + v_off;
            const int k0 = kt * TW_K;
#pragma unroll
            for (int i = 0; i < NCH; ++i)
                if (pt + i * TW_NPROD < S * Sh::VR * TW_KQ)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sb + dsto[i]), "l"(srcp[i] + k0),
                                 "r"(nbytes[i]));
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(tw_smem(&full[b])) : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    // ---- epilogue (all warps) once every product is in tensor memory
    __syncwarp();
    // idle threads poll gently
    const bool ok = !s_fail && mbar_wait_bounded(tw_smem(&done), 0, kWaitLimitNs, 64);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (__syncthreads_and(ok)) {
        const int q4 = warp & 3, half = warp >> 2;
        if (TM) {
            // lane = table row, columns = pairs
            const int i = row0 + q4 * 32 + lane;
            const int row_e = s_rowe[q4 * 32 + lane];
            for (int c0 = half * (NB / 2); c0 < (half + 1) * (NB / 2); c0 += 8) {
                uint32_t r[S][8];
#pragma unroll
                for (int d = 0; d < S; ++d) {
                    const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(d * NB + c0);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                                 : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3]), "=r"(r[d][4]),
                                   "=r"(r[d][5]), "=r"(r[d][6]), "=r"(r[d][7])
                                 : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (i < a.M) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = c0 + j;
                        if (s_pdst[n] < 0) continue;
                        float acc[S];
#pragma unroll
                        for (int d = 0; d < S; ++d) acc[d] = __uint_as_float(r[d][j]);
                        const double val = slice_output<S>(acc, s_ps[n], row_e);
                        double *o = a.out + s_pdst[n] + i;
                        if (a.add) atomicAdd(o, val);
                        else *o = val;
                    }
                }
            }
        } else {
            // lane = pair, columns = table rows; a warp-private buffer makes the
            // atomics row-contiguous (lane l: row l % 8 of pair l / 8 + 4 it)
            double *xb = reinterpret_cast<double *>(wsm) + (size_t)warp * 32 * 9;   // stages no longer read
            const int p = q4 * 32 + lane;
            for (int c0 = half * (NB / 2); c0 < (half + 1) * (NB / 2); c0 += 8) {
                uint32_t r[S][8];
#pragma unroll
                for (int d = 0; d < S; ++d) {
                    const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(d * NB + c0);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                                 : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3]), "=r"(r[d][4]),
                                   "=r"(r[d][5]), "=r"(r[d][6]), "=r"(r[d][7])
                                 : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float acc[S];
#pragma unroll
                    for (int d = 0; d < S; ++d) acc[d] = __uint_as_float(r[d][j]);
                    xb[lane * 9 + j] = slice_output<S>(acc, s_ps[p], s_rowe[c0 + j]);
                }
                __syncwarp();
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int pl = it * 4 + (lane >> 3), j = lane & 7;
                    const int64_t dst = s_pdst[q4 * 32 + pl];
                    const int row = row0 + c0 + j;
                    if (dst >= 0 && row < a.M) {
                        double *o = a.out + dst + row;
                        if (a.add) atomicAdd(o, xb[pl * 9 + j]);
                        else *o = xb[pl * 9 + j];
                    }
                }
                __syncwarp();
            }
        }
    } else if (tid == 0) {
        set_status(a.status, VPX_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(Sh::TMEM_COLS));
    }
}

// ------------------------------------------------------------------ host

// Which mixed-form passes run here (0: none, 1: table rows on M): every pass
// with an inner dimension in whole 32-deep stages.
// The far-field tables (2(p+1) rows, 56 at p = 27) take one 128-row block,
// whose copies read up to 127 rows past the last chunk into the interleaved
// table's padding; rows >= M are computed and dropped.
static int ws_kind(const GemmPass &g) {
    if (!g.tslices || g.Kpad % TW_K != 0) return 0;
    return 1;
}

// the table slices re-laid as [tab][slice][Kpad/8][Mpad][8] (plus one row block
// of padding, so that a last row block running past Mpad stays inside)
__global__ void k_interleave_table(const uint16_t *ts, int ntab, int Mpad, int Kpad, uint16_t *ti) {
    const size_t n = (size_t)ntab * kSlicesS * Mpad * Kpad;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t ts_row = e / Kpad;   // (tab, s, row)
        const int k = (int)(e % Kpad), row = (int)(ts_row % Mpad);
        const size_t tsl = ts_row / Mpad;   // tab * S + s
        ti[((tsl * (Kpad / 8) + k / 8) * Mpad + row) * 8 + (k % 8)] = ts[e];
    }
}

void gemm_ws_prepare(GemmPass &g) {
    const int kind = ws_kind(g);
    if (!kind) return;
    const size_t n = (size_t)g.ntab * kSlicesS * g.Mpad * g.Kpad;
    uint16_t *ti = dev_alloc<uint16_t>(n + (size_t)TW_M * 8);
    VPX_CUDA(cudaMemset(ti, 0, (n + (size_t)TW_M * 8) * sizeof(uint16_t)));
    k_interleave_table<<<1024, 256>>>(g.tslices, g.ntab, g.Mpad, g.Kpad, ti);
    VPX_LAUNCH("k_interleave_table");
    VPX_CUDA(cudaDeviceSynchronize());
    g.tint = ti;
    g.ws_kind = kind;
}

template <bool TM, int S, int NB>
static void ws_attr() {
    VPX_CUDA(cudaFuncSetAttribute(k_gemm_ws<TM, S, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)WsShape<TM, S, NB>::SMEM));
}

void gemm_ws_prepare_device() {
    ws_attr<true, kSlicesS, kWsTileN>();
}

bool gemm_ws_eligible(const GemmPass &g, const VecSet &vs) {
    return g.ws_kind != 0 && vs.slices != nullptr && vs.kpad == g.Kpad;
}

void gemm_ws_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s) {
    WsArgs a;
    a.M = g.M;
    a.Mpad = g.Mpad;
    a.Kpad = g.Kpad;
    a.nvec = vs.nvec;
    a.texpo = g.texpo;
    a.pairs = g.pairs;
    a.vslices = vs.slices;
    a.vexpo = vs.expo;
    a.out = out;
    a.ldo = ldo;
    a.add = g.add;
    a.status = g.status;
    a.tint = g.tint;
    cudaStream_t st = (cudaStream_t)s;
    const dim3 rb(1, (g.M + TW_M - 1) / TW_M, nrhs);
    if (g.n_tiles_w == 0) return;
    a.tiles = g.tiles_w;
    launch_pdl(k_gemm_ws<true, kSlicesS, kWsTileN>, dim3(g.n_tiles_w, rb.y, rb.z), dim3(TW_THREADS),
               WsShape<true, kSlicesS, kWsTileN>::SMEM, st, a);
    VPX_LAUNCH("k_gemm_ws");
}

}  // namespace vpx
