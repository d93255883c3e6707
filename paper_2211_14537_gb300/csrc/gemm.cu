// gemm.cu -- the grouped table GEMM (gemm.cuh): FP64 engine, slicing of
// vectors and tables for the exact-slice engines, pass setup and dispatch.
//
// FP64 form: 64 x 64 output tile per CTA, 4 x 4 FP64 register tile per thread,
// 16-deep k stages in shared memory.
//
// Mixed form (exact bf16 slices): each table row i is scaled by 2^-e_i with
// max|row| < 2^(e_i - 1) and split into S = 4 (near field) or 5 (far field)
// integer slices of 8 bits, balanced base-256 digits of magnitude <= 128;
// each source vector likewise with its own exponent (slice_math.cuh).  A
// product of two slices is an integer of magnitude <= 2^14; per inner index
// the products of order d sum to at most (d + 1) 2^14, so every order sum is
// exact in the tensor cores' fp32 accumulation while K (d + 1) <= 1024
// (slice_math.cuh).  The orders are combined in int64 and scaled by
// scale_p 2^{e_i + e_v - 16 - 8(S-1)}; the truncation error is about
// 2^-(8S-1) relative to max|row| max|vector|.  Two engines run it:
// warp-specialised tcgen05 with TMA and TMEM accumulators (gemm_ws.cu) and
// mma.sync with tables in fragment order (gemm_frag.cu); a double-float
// engine on the fp32 pipes (gemm_rows.cu) takes the short level chains.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "dev_common.cuh"
#include "gemm.cuh"
#include "slice_math.cuh"

namespace vpx {

// ------------------------------------------------------------ FP64 engine

constexpr int G_M = 64, G_K = 16;

// One CTA: G_M table rows x GN pairs, 256 threads as TY x TX with RI rows and NJ
// pairs each.  GN = 64 for passes that fill the GPU; GN = 8 for the small ones
// (the level chains), whose few wide tiles would leave most SMs idle at the
// FP64 rate.  Each output sums over k in the same order for every GN.
template <int GN>
__global__ void __launch_bounds__(256) k_gemm_fp64(int M, int Kd, const double *tab, const GTile *tiles,
                                                   const GPair *pairs, const double *vbase, int64_t vld,
                                                   int vstride, double *out, int64_t ldo, int add) {
    pdl_entry();
    constexpr int TX = GN < 16 ? GN : 16, TY = 256 / TX, RI = G_M / TY, NJ = GN / TX;
    static_assert(TX * TY == 256 && RI * TY == G_M && NJ * TX == GN, "thread layout");
    __shared__ double As[G_K][G_M + 1];
    __shared__ double Bs[G_K][GN + 1];
    const GTile tile = tiles[blockIdx.x];
    const int m0 = blockIdx.y * G_M, rhs = blockIdx.z;
    const double *A = tab + (size_t)tile.tab * M * Kd;
    const double *V = vbase + rhs * vld;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    double acc[RI][NJ] = {};
    for (int k0 = 0; k0 < Kd; k0 += G_K) {
        for (int e = threadIdx.x; e < G_M * G_K; e += 256) {
            int r = e / G_K, k = e % G_K;
            As[k][r] = (m0 + r < M && k0 + k < Kd) ? A[(size_t)(m0 + r) * Kd + k0 + k] : 0.0;
        }
        for (int e = threadIdx.x; e < GN * G_K; e += 256) {
            int n = e / G_K, k = e % G_K;
            Bs[k][n] = (n < tile.count && k0 + k < Kd)
                           ? V[(int64_t)pairs[tile.first + n].src * vstride + k0 + k]
                           : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < G_K; ++k) {
            double ar[RI], br[NJ];
#pragma unroll
            for (int i = 0; i < RI; ++i) ar[i] = As[k][ty * RI + i];
#pragma unroll
            for (int j = 0; j < NJ; ++j) br[j] = Bs[k][tx + TX * j];
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[i][j] += ar[i] * br[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        int n = tx + TX * j;
        if (n >= tile.count) continue;
        const GPair pr = pairs[tile.first + n];
        double *o = out + rhs * ldo + pr.dst;
#pragma unroll
        for (int i = 0; i < RI; ++i) {
            int r = m0 + ty * RI + i;
            if (r >= M) continue;
            if (add) atomicAdd(o + r, pr.scale * acc[i][j]);
            else o[r] = pr.scale * acc[i][j];
        }
    }
}

// ------------------------------------------------------------ slicing

// the slicing exponent of a table row (as slice_expo_of_bits): amax < 2^(e-1)
__device__ __host__ inline int slice_expo(double amax) {
    if (!(amax > 0.0)) return 0;
    int e;
    frexp(amax, &e);
    return e + 1;
}

// One warp per (vector, rhs): exponent and slices (slice_math.cuh), zero padded to Kpad.

__global__ void k_slice_vec(const double *vbase, int64_t vld, int vstride, int first, int count, int Kd, int Kpad,
                            int nvec, uint16_t *slices, int32_t *expo) {
    pdl_entry();
    const int vi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31, rhs = blockIdx.y;
    if (vi >= count) return;
    const int v = first + vi;
    const double *x = vbase + rhs * vld + (int64_t)v * vstride;
    double xv[kSliceMaxPerLane];
    uint64_t mb = 0;
#pragma unroll
    for (int q = 0; q < kSliceMaxPerLane; ++q) {   // all loads first
        const int j = lane + 32 * q;
        xv[q] = (j < Kd) ? x[j] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kSliceMaxPerLane; ++q) {
        const uint64_t t = slice_abs_bits(xv[q]);
        mb = t > mb ? t : mb;
    }
    const int e = slice_warp_expo(mb);
    uint16_t *out = slices + ((size_t)rhs * nvec + v) * kSlicesS * Kpad;
#pragma unroll
    for (int q = 0; q < kSliceMaxPerLane; ++q) {
        const int j = lane + 32 * q;
        if (j >= Kpad) break;
        uint16_t d[kSlicesS];
        slice_digits(slice_fixed_point(xv[q], e), d);
#pragma unroll
        for (int k = 0; k < kSlicesS; ++k) out[(size_t)k * Kpad + j] = d[k];
    }
    if (lane == 0) expo[(size_t)rhs * nvec + v] = e;
}

// ------------------------------------------------------------------ host

void gemm_pass_set_pairs(GemmPass &g, std::vector<std::pair<int, GPair>> &tagged, int frag_np) {
    std::stable_sort(tagged.begin(), tagged.end(),
                     [](const std::pair<int, GPair> &x, const std::pair<int, GPair> &y) { return x.first < y.first; });
    std::vector<GPair> pr;
    std::vector<GTile> tl, tf, tfa, tr, tw;
    const size_t npf = frag_np == 8 || frag_np == 32 ? (size_t)frag_np : tagged.size() >= (size_t)kFragBigPass ? 32 : 8;
    const size_t npa = npf == 8 ? 32 : 8;
    size_t i = 0;
    while (i < tagged.size()) {
        size_t j = i;
        while (j < tagged.size() && tagged[j].first == tagged[i].first) ++j;
        const int32_t base = (int32_t)pr.size();
        for (size_t k = i; k < j; k += kGemmTileN)
            tl.push_back({tagged[i].first, base + (int32_t)(k - i), (int32_t)std::min<size_t>(kGemmTileN, j - k), 0});
        for (size_t k = i; k < j; k += kWsTileN)
            tw.push_back({tagged[i].first, base + (int32_t)(k - i), (int32_t)std::min<size_t>(kWsTileN, j - k), 0});
        for (size_t k = i; k < j; k += npf)
            tf.push_back({tagged[i].first, base + (int32_t)(k - i), (int32_t)std::min<size_t>(npf, j - k), 0});
        for (size_t k = i; k < j; k += npa)
            tfa.push_back({tagged[i].first, base + (int32_t)(k - i), (int32_t)std::min<size_t>(npa, j - k), 0});
        for (size_t k = i; k < j; k += kRowsTileN)
            tr.push_back({tagged[i].first, base + (int32_t)(k - i), (int32_t)std::min<size_t>(kRowsTileN, j - k), 0});
        for (size_t k = i; k < j; ++k) pr.push_back(tagged[k].second);
        i = j;
    }
    // largest tiles first: CTAs start in tile order, so a pass of more than one
    // wave ends with its smallest tiles (stable: full tiles keep their table
    // order).  The row engine pairs tile i with pair i and keeps its order.
    auto by_count = [](const GTile &x, const GTile &y) { return x.count > y.count; };
    for (std::vector<GTile> *v : {&tl, &tf, &tfa, &tw}) std::stable_sort(v->begin(), v->end(), by_count);
    g.h_pairs = pr;
    g.n_pairs = (int)pr.size();
    g.n_tiles = (int)tl.size();
    g.n_tiles_f = (int)tf.size();
    g.n_tiles_r = (int)tr.size();
    g.n_tiles_w = (int)tw.size();
    g.np_f = (int)npf;
    g.n_tiles_f_alt = (int)tfa.size();
    g.np_f_alt = (int)npa;
    g.tiles_f_alt = dev_upload(tfa);
    g.pairs = dev_upload(pr);
    g.tiles = dev_upload(tl);
    g.tiles_f = dev_upload(tf);
    g.tiles_r = dev_upload(tr);
    g.tiles_w = dev_upload(tw);
}

static uint16_t bf16_bits_exact(double q) {
    // q is an integer with |q| <= 128: exact in bf16
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
    // the same slices in mma.sync m16n8k16 A-fragment order: lane (g, q) of the
    // fragment (m16 block mb, k16 block kb) holds rows mb*16+g, +8 and columns
    // kb*16+2q, +1, +8, +9, two bf16 per 32-bit register (lower column low)
    const int MB = g.Mpad / 16, KB = g.Kpad / 16;
    std::vector<uint32_t> fr((size_t)ntab * kSlicesS * MB * KB * 32 * 4);
    auto at = [&](int t, int s, int r, int c) -> uint32_t {
        return sl[(((size_t)t * kSlicesS + s) * g.Mpad + r) * g.Kpad + c];
    };
    size_t o = 0;
    for (int t = 0; t < ntab; ++t)
        for (int s = 0; s < kSlicesS; ++s)
            for (int mb = 0; mb < MB; ++mb)
                for (int kb = 0; kb < KB; ++kb)
                    for (int lane = 0; lane < 32; ++lane) {
                        const int r0 = mb * 16 + (lane >> 2), c0 = kb * 16 + 2 * (lane & 3);
                        fr[o++] = at(t, s, r0, c0) | at(t, s, r0, c0 + 1) << 16;
                        fr[o++] = at(t, s, r0 + 8, c0) | at(t, s, r0 + 8, c0 + 1) << 16;
                        fr[o++] = at(t, s, r0, c0 + 8) | at(t, s, r0, c0 + 9) << 16;
                        fr[o++] = at(t, s, r0 + 8, c0 + 8) | at(t, s, r0 + 8, c0 + 9) << 16;
                    }
    g.tfrag = dev_upload(fr);
}

void gemm_rows_prepare(const GemmPass &g);

bool gemm_pass_use_rows(GemmPass &g, const std::vector<double> &tab) {
    if (g.M > 96 || (size_t)g.Kd * g.M * 8 > 160 * 1024) return false;
    for (const GPair &p : g.h_pairs) {
        int e = 0;
        if (std::frexp(p.scale, &e) != 0.5) return false;
    }
    const size_t ts = ((size_t)g.Kd * g.M + 1) / 2 * 2;   // table stride: a multiple of 16 bytes
    std::vector<float2> t((size_t)g.ntab * ts, make_float2(0.f, 0.f));
    for (int q = 0; q < g.ntab; ++q)
        for (int i = 0; i < g.M; ++i)
            for (int k = 0; k < g.Kd; ++k) {
                const double v = tab[((size_t)q * g.M + i) * g.Kd + k];
                const float h = (float)v;
                t[q * ts + (size_t)k * g.M + i] = make_float2(h, (float)(v - (double)h));
            }
    g.tdfT = dev_upload(t);
    gemm_rows_prepare(g);
    return true;
}

void gemm_pass_free(GemmPass &g) {
    if (g.owns_tables) {
        dev_free(g.tab);
        dev_free(g.tslices);
        dev_free(g.texpo);
        dev_free(g.tfrag);
        dev_free(g.tdfT);
        dev_free(g.tint);
    }
    g.tab = nullptr;
    g.tslices = nullptr;
    g.texpo = nullptr;
    g.tfrag = nullptr;
    g.tdfT = nullptr;
    g.tint = nullptr;
    dev_free(g.pairs);
    dev_free(g.tiles);
    dev_free(g.tiles_f);
    dev_free(g.tiles_f_alt);
    dev_free(g.tiles_r);
    dev_free(g.tiles_w);
    g.n_pairs = g.n_tiles = g.n_tiles_f = g.n_tiles_f_alt = g.n_tiles_r = g.n_tiles_w = 0;
}

void gemm_pass_view(GemmPass &v, const GemmPass &base) {
    v = GemmPass();
    v.M = base.M;
    v.Kd = base.Kd;
    v.Kpad = base.Kpad;
    v.Mpad = base.Mpad;
    v.ntab = base.ntab;
    v.add = base.add;
    v.status = base.status;
    v.tab = base.tab;
    v.tslices = base.tslices;
    v.texpo = base.texpo;
    v.tfrag = base.tfrag;
    v.tdfT = base.tdfT;
    v.tint = base.tint;
    v.ws_kind = base.ws_kind;
    v.engine = base.engine;
    v.owns_tables = false;
}

GemmChoice gemm_choice(const GemmPass &g) { return GemmChoice{g.engine, g.np_f}; }

void gemm_set_choice(GemmPass &g, GemmChoice c) {
    g.engine = c.engine;
    if (c.np_f != 0 && c.np_f != g.np_f && c.np_f == g.np_f_alt) {   // np_f 0: keep the current width
        std::swap(g.tiles_f, g.tiles_f_alt);
        std::swap(g.n_tiles_f, g.n_tiles_f_alt);
        std::swap(g.np_f, g.np_f_alt);
    }
}

static thread_local std::vector<GemmCall> *t_recorder = nullptr;

bool pdl_enabled() {
    static const bool on = getenv("VPX_NO_PDL") == nullptr;
    return on;
}

void gemm_set_recorder(std::vector<GemmCall> *rec) { t_recorder = rec; }

int &launch_priority() {
    static thread_local int prio = kNoPriority;
    return prio;
}

static void priority_range(int &least, int &greatest) {
    static int l = 0, g = 0, done = 0;
    if (!done) {
        VPX_CUDA(cudaDeviceGetStreamPriorityRange(&l, &g));
        done = 1;
    }
    least = l;
    greatest = g;
}

int priority_greatest() {
    if (getenv("VPX_NO_PRIORITY")) return kNoPriority;
    int l, g;
    priority_range(l, g);
    return g;
}

int priority_least() {
    if (getenv("VPX_NO_PRIORITY")) return kNoPriority;
    int l, g;
    priority_range(l, g);
    return l;
}

bool gemm_frag_eligible(const GemmPass &g, const VecSet &vs);
void gemm_rows_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s);
bool gemm_ws_eligible(const GemmPass &g, const VecSet &vs);
void gemm_ws_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s);
void gemm_frag_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, void *s);

void gemm_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, bool mixed, void *sv) {
    if (g.n_tiles == 0) return;
    cudaStream_t s = (cudaStream_t)sv;
    if (!mixed) {
        // 64-pair tiles when they give at least two CTAs per SM, else the 8-pair
        // tiles of the fragment engine (one of its two widths is 8)
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            VPX_CUDA(cudaGetDevice(&dev));
            VPX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        }
        const int mb = (g.M + G_M - 1) / G_M;
        const GTile *t8 = g.np_f == 8 ? g.tiles_f : g.tiles_f_alt;
        const int n8 = g.np_f == 8 ? g.n_tiles_f : g.n_tiles_f_alt;
        if ((int64_t)g.n_tiles * mb * nrhs < 2 * sms && t8 && n8 > 0)
            launch_pdl(k_gemm_fp64<8>, dim3(n8, mb, nrhs), dim3(256), 0, s, g.M, g.Kd, g.tab, (const GTile *)t8,
                       (const GPair *)g.pairs, vs.base, vs.ld, vs.stride, out, ldo, g.add);
        else
            launch_pdl(k_gemm_fp64<64>, dim3(g.n_tiles, mb, nrhs), dim3(256), 0, s, g.M, g.Kd, g.tab,
                       (const GTile *)g.tiles, (const GPair *)g.pairs, vs.base, vs.ld, vs.stride, out, ldo, g.add);
        VPX_LAUNCH("k_gemm_fp64");
        return;
    }
    if (g.tdfT) {
        gemm_rows_run(g, vs, out, ldo, nrhs, sv);
        return;
    }
    if (t_recorder) t_recorder->push_back(GemmCall{const_cast<GemmPass *>(&g), vs, out, ldo, nrhs});
    // read per call, so that a test can compare the engines: VPX_NO_TC keeps
    // every pass off tcgen05, VPX_TC_ALL puts every eligible pass on it
    const bool no_tc = getenv("VPX_NO_TC") != nullptr, all_tc = getenv("VPX_TC_ALL") != nullptr;
    if (!no_tc && (g.engine == 0 || all_tc) && gemm_ws_eligible(g, vs)) {
        gemm_ws_run(g, vs, out, ldo, nrhs, sv);
        return;
    }
    if (!gemm_frag_eligible(g, vs)) fail(VPX_ERR_ARG, "no exact-slice engine covers this pass shape");
    gemm_frag_run(g, vs, out, ldo, nrhs, sv);
}

void slice_vectors(const VecSet &vs, int first, int count, int Kd, int Kpad, int nrhs, void *sv) {
    if (count <= 0) return;
    if (Kpad > 32 * kSliceMaxPerLane) fail(VPX_ERR_ARG, "slice_vectors: vectors longer than 256");
    launch_pdl(k_slice_vec, dim3((count + 7) / 8, nrhs), dim3(256), 0, (cudaStream_t)sv, vs.base, vs.ld, vs.stride, first, count, Kd,
                                                                            Kpad, vs.nvec, vs.slices, vs.expo);
    VPX_LAUNCH("k_slice_vec");
}

}  // namespace vpx
