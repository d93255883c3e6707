// chain.cu -- the two level chains of the box FMM (Section 4.1), each as ONE
// persistent launch driven by a work queue in device memory, in place of one
// launch per level:
//
//   upward   M2M: a box's multipole is final once every non-zero child has
//            been translated into it.  Every non-zero box at level >= 3 is
//            translated once; the non-zero leaves are ready at the start.
//            Processing box c adds T_pos(c) mp[c] into mp[parent(c)] (atomic:
//            several children add into one parent).
//   downward L2L: a box's local expansion is final once its parent's is
//            (every other contribution -- M2L, list i+, the constant terms --
//            is complete before the launch).  Every box at level >= 3 is
//            processed once; those at level 3 are ready at the start.
//            Processing box c adds T_pos(c) lo[parent(c)] into lo[c] (its only
//            writer in the launch).
//
// T_pos is the translation of the child position pos in 0..3 (the same real
// 2(p+1) x 2(p+1) tables as the per-level passes) in complex form, P x P with
// P = p + 1, read from global memory (L2-resident), each row summed over its
// non-zero column range only: M2M is lower and L2L upper triangular in these
// variables.  The mixed form computes in double-float (df32.cuh) on the fp32
// pipes, the FP64 form in FP64.
//
// Scheduling.  Upward, the CTA whose translation completes a parent's count
// goes on with that parent itself, so a CTA claims only the initially ready
// leaves (a fixed list: a claim never waits) and climbs as far as it
// completes.  Downward, a CTA goes on with the first child of the box it
// processed and queues the other three: a claim counter hands out slots in
// order, slot h < n0 holding the h-th box of level 3 and slot h >= n0 the
// (h - n0)-th queued box (0 until written).  A CTA claims a slot, waits until
// it is written, and processes from there.  No CTA waits while it holds a box,
// and every queued-but-unwritten slot belongs to a box whose parent is being
// processed by a running CTA, so the waits end whether or not every CTA of
// the grid is resident at once.  Each wait is bounded in wall-clock time
// besides: a timeout latches VPX_ERR_TIMEOUT and the CTA leaves.  The queue
// state (claim and push counters, per-box counts, slots) is one zeroed block
// per launch.
//
// The mixed form runs the warp-granular kernel k_wchain below (one warp per
// box).  On the L-shape at p = 27 its chains take 73 us (up) and 81 us (down)
// against 98 and 100 us for the CTA-per-box kernel and 71 and 79 us for one
// launch per level: a level costs about 6 us either way, set by the memory
// round trips of one box (its atomics and fence, the parent's counter, the
// parent's load) rather than by launches.  So the mixed form's default stays
// one launch per level; both kernels remain selectable.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "bulk.cuh"
#include "dev_common.cuh"
#include "df32.cuh"

namespace vpx {

constexpr int CH_THREADS = 256;   // one box at a time per CTA; rows x column groups, several CTAs per SM

struct ChainArgs {
    int P, nrhs, n_slots, n0, G;  // slots: ready boxes at the start + boxes queued (downward); G: column groups per row
    int64_t ldm;                  // doubles per right-hand side of the expansion arrays
    const int32_t *items0;        // [n0] initially ready boxes
    const int2 *up_of;            // per box: (parent, position 0..3 among its siblings)
    const int32_t *child0, *need; // per box; need: non-zero children to wait for (upward, 0: not translated on)
    const void *tab;              // [4][P][P] complex: double2 (FP64 form) or float4 hi/lo pairs (mixed form)
    const int16_t *krange;        // [4][P][2] non-zero column range of every row
    int *ws;                      // [2 + n_boxes + n_slots]: claim, push, per-box counts, queued slots (box + 1)
    int n_boxes;
    double *x;                    // expansions: mp (upward) or lo (downward), [rhs][box][2P]
    int *status;
};

__device__ inline int ld_acquire_int(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0: claim the next slot and wait for its box; -1 = no items left, -2 = gave up
__device__ inline int chain_claim(const ChainArgs &a) {
    const int h = atomicAdd(a.ws, 1);
    if (h >= a.n_slots) return -1;
    if (h < a.n0) return a.items0[h];
    const int *slot = a.ws + 2 + a.n_boxes + (h - a.n0);
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {
        const int v = ld_acquire_int(slot);
        if (v > 0) {
            __threadfence();
            return v - 1;
        }
        if ((it & 63u) == 63u && global_ns() - t0 > kWaitLimitNs) break;
        __nanosleep(32);
    }
    set_status(a.status, VPX_ERR_TIMEOUT);
    return -2;
}

__device__ inline void chain_push(const ChainArgs &a, int box) {
    const int s = atomicAdd(a.ws + 1, 1);
    if (s < a.n_slots - a.n0) atomicExch(a.ws + 2 + a.n_boxes + s, box + 1);
}

// table entries per thread and box, ceil(P / G): at most 8 for P <= 45, 16 for P <= 64

// One CTA processes one box at a time; the tables stay in global memory (a
// few hundred KB, L2-resident), so the CTA needs little shared memory and
// several fit on an SM beside the near-field kernel of the other stream.
// Thread t < P G takes row t / G and the columns klo + (t % G) + G j; it loads
// all its table entries of the box at once, then computes.  Upward, CTA b
// starts from leaves b, b + grid, ... (a claim never waits, so no counter).
template <bool DF, bool UP, int CH_NK>
__global__ void __launch_bounds__(CH_THREADS) k_chain(ChainArgs a) {
    pdl_entry();
    typedef typename std::conditional<DF, float4, double2>::type E;
    __shared__ __align__(16) E s_vec[kMaxP];                 // the source expansion
    __shared__ __align__(16) E s_part[CH_THREADS];           // partial sums (re, im) per thread
    __shared__ int16_t s_kr[4 * kMaxP * 2];                  // non-zero column ranges of the four tables
    __shared__ int s_item;
    const int P = a.P, G = a.G, tid = threadIdx.x;
    const int row = tid / G, g = tid % G;
    const bool act = row < P;
    for (int i = tid; i < 4 * P * 2; i += CH_THREADS) s_kr[i] = a.krange[i];
    int c = -1;          // the box in hand; -1: claim the next slot
    int next_leaf = blockIdx.x;
    for (;;) {
        __syncthreads();   // the previous box's reads of s_vec, s_part and s_item are done
        if (c < 0) {
            if (UP) {
                c = next_leaf < a.n0 ? a.items0[next_leaf] : -1;
                next_leaf += gridDim.x;
            } else {
                if (tid == 0) s_item = chain_claim(a);
                __syncthreads();
                c = s_item;
            }
            if (c < 0) break;
        }
        const int2 up = a.up_of[c];
        const int par = up.x, pos = up.y;
        const int src = UP ? c : par, dst = UP ? par : c;
        int klo = 0, khi = -1;
        if (act) {
            klo = s_kr[(pos * P + row) * 2];
            khi = s_kr[(pos * P + row) * 2 + 1];
        }
        const E *T = reinterpret_cast<const E *>(a.tab) + ((size_t)pos * P + (act ? row : 0)) * P;
        E tv[CH_NK];
#pragma unroll
        for (int j = 0; j < CH_NK; ++j) {
            const int k = klo + g + j * G;
            if (k <= khi) tv[j] = __ldg(T + k);
        }
        for (int r = 0; r < a.nrhs; ++r) {
            const double *xs = a.x + r * a.ldm + (int64_t)src * 2 * P;
            if (tid < P) {
                const double re = __ldcg(xs + 2 * tid), im = __ldcg(xs + 2 * tid + 1);
                if (DF) {
                    const df32 hr = df_split_bits(re), hi = df_split_bits(im);
                    reinterpret_cast<float4 *>(s_vec)[tid] = make_float4(hr.hi, hr.lo, hi.hi, hi.lo);
                } else {
                    reinterpret_cast<double2 *>(s_vec)[tid] = make_double2(re, im);
                }
            }
            __syncthreads();
            if (DF) {
                df32 sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll
                for (int j = 0; j < CH_NK; ++j) {
                    const int k = klo + g + j * G;
                    if (k > khi) break;
                    const float4 t = reinterpret_cast<const float4 &>(tv[j]);
                    const float4 v = reinterpret_cast<const float4 *>(s_vec)[k];
                    df_mac(sr, df32{t.x, t.y}, df32{v.x, v.y});
                    df_mac(sr, df32{-t.z, -t.w}, df32{v.z, v.w});
                    df_mac(si, df32{t.x, t.y}, df32{v.z, v.w});
                    df_mac(si, df32{t.z, t.w}, df32{v.x, v.y});
                }
                sr = df_norm(sr);
                si = df_norm(si);
                reinterpret_cast<float4 *>(s_part)[tid] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
            } else {
                double sr = 0.0, si = 0.0;
#pragma unroll
                for (int j = 0; j < CH_NK; ++j) {
                    const int k = klo + g + j * G;
                    if (k > khi) break;
                    const double2 t = reinterpret_cast<const double2 &>(tv[j]);
                    const double2 v = reinterpret_cast<const double2 *>(s_vec)[k];
                    sr = fma(t.x, v.x, fma(-t.y, v.y, sr));
                    si = fma(t.x, v.y, fma(t.y, v.x, si));
                }
                reinterpret_cast<double2 *>(s_part)[tid] = make_double2(sr, si);
            }
            __syncthreads();
            if (tid < P) {
                const int l = tid;
                double out_re, out_im;
                if (DF) {
                    df32 sr{0.f, 0.f}, si{0.f, 0.f};
                    for (int q = 0; q < G; ++q) {
                        const float4 v = reinterpret_cast<const float4 *>(s_part)[l * G + q];
                        sr = df_add(sr, df32{v.x, v.y});
                        si = df_add(si, df32{v.z, v.w});
                    }
                    out_re = df_to_f64_scaled(sr, 0);
                    out_im = df_to_f64_scaled(si, 0);
                } else {
                    out_re = out_im = 0.0;
                    for (int q = 0; q < G; ++q) {
                        const double2 v = reinterpret_cast<const double2 *>(s_part)[l * G + q];
                        out_re += v.x;
                        out_im += v.y;
                    }
                }
                double *xd = a.x + r * a.ldm + (int64_t)dst * 2 * P + 2 * l;
                if (UP) {
                    atomicAdd(xd, out_re);
                    atomicAdd(xd + 1, out_im);
                } else {
                    xd[0] = __ldcg(xd) + out_re;
                    xd[1] = __ldcg(xd + 1) + out_im;
                }
            }
            if (r + 1 < a.nrhs) __syncthreads();   // s_vec and s_part are rewritten for the next column
        }
        __threadfence();       // this box's results are visible before anything goes on from them
        __syncthreads();
        if (tid == 0) {
            int next = -1;
            if (UP) {          // the child that completes its parent's count goes on with the parent
                const int nd = a.need[par];
                if (nd > 0 && atomicAdd(a.ws + 2 + par, 1) == nd - 1) {
                    __threadfence();
                    next = par;
                }
            } else {           // on with the first child; the other three to the queue
                const int ch = a.child0[c];
                if (ch >= 0) {
                    for (int k = 1; k < 4; ++k) chain_push(a, ch + k);
                    next = ch;
                }
            }
            s_item = next;
        }
        __syncthreads();
        c = s_item;
    }
}

// ---------------------------------------------------------- warp-granular form

// The mixed form's chains with ONE WARP per box instead of one CTA: the
// schedule above at warp granularity (a warp that completes a parent goes on
// with it; downward, a warp goes on with a first child and queues the rest),
// so a CTA of CW_WARPS warps carries as many boxes at once.  The four tables
// stay in shared memory, each row packed over its non-zero column range
// (M2M is lower and L2L upper triangular, so half of P x P); lane l computes
// rows l and l + 32.  Every box still costs the same double-float operations
// as in k_chain, summed in column order per row.
constexpr int CW_WARPS = 8, CW_THREADS = 32 * CW_WARPS;

struct WChainArgs {
    int P, nrhs, n_slots, n0, n_packed;
    int64_t ldm;
    const int32_t *items0;
    const int2 *up_of;
    const int32_t *child0, *need;
    const float4 *tabp;           // packed rows: (re hi, re lo, im hi, im lo) over each row's column range
    const int32_t *roff;          // [4][P] start of every row in tabp
    const int16_t *krange;        // [4][P][2]
    int *ws;
    int n_boxes;
    double *x;
    int *status;
};

// lane 0: claim the next slot and wait for its box (as chain_claim)
__device__ inline int wchain_claim(const WChainArgs &a) {
    const int h = atomicAdd(a.ws, 1);
    if (h >= a.n_slots) return -1;
    if (h < a.n0) return a.items0[h];
    const int *slot = a.ws + 2 + a.n_boxes + (h - a.n0);
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {
        const int v = ld_acquire_int(slot);
        if (v > 0) {
            __threadfence();
            return v - 1;
        }
        if ((it & 63u) == 63u && global_ns() - t0 > kWaitLimitNs) break;
        __nanosleep(32);
    }
    set_status(a.status, VPX_ERR_TIMEOUT);
    return -2;
}

template <bool UP>
__global__ void __launch_bounds__(CW_THREADS) k_wchain(WChainArgs a) {
    pdl_entry();
    extern __shared__ __align__(16) float4 cw_sm[];
    const int P = a.P, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *s_tab = cw_sm;                                           // [n_packed]
    float4 *s_x = cw_sm + a.n_packed + warp * P;                     // [CW_WARPS][P]: the source expansion
    int *s_off = reinterpret_cast<int *>(cw_sm + a.n_packed + CW_WARPS * P);   // [4][P]
    int16_t *s_kr = reinterpret_cast<int16_t *>(s_off + 4 * P);      // [4][P][2]
    for (int i = threadIdx.x; i < a.n_packed; i += CW_THREADS) s_tab[i] = a.tabp[i];
    for (int i = threadIdx.x; i < 4 * P; i += CW_THREADS) s_off[i] = a.roff[i];
    for (int i = threadIdx.x; i < 8 * P; i += CW_THREADS) s_kr[i] = a.krange[i];
    __syncthreads();
    const int gw = blockIdx.x * CW_WARPS + warp, nw = gridDim.x * CW_WARPS;
    int next_leaf = gw;
    int c = -1;
    for (;;) {
        if (c < 0) {
            if (UP) {
                c = next_leaf < a.n0 ? a.items0[next_leaf] : -1;
                next_leaf += nw;
            } else {
                int v = 0;
                if (lane == 0) v = wchain_claim(a);
                c = __shfl_sync(0xffffffffu, v, 0);
            }
            if (c < 0) break;
        }
        const int2 up = a.up_of[c];
        const int par = up.x, pos = up.y;
        const int src = UP ? c : par, dst = UP ? par : c;
        for (int r = 0; r < a.nrhs; ++r) {
            const double *xs = a.x + r * a.ldm + (int64_t)src * 2 * P;
            for (int k = lane; k < P; k += 32) {
                const df32 hr = df_split_bits(__ldcg(xs + 2 * k)), hi = df_split_bits(__ldcg(xs + 2 * k + 1));
                s_x[k] = make_float4(hr.hi, hr.lo, hi.hi, hi.lo);
            }
            __syncwarp();
            for (int l = lane; l < P; l += 32) {
                const int klo = s_kr[(pos * P + l) * 2], khi = s_kr[(pos * P + l) * 2 + 1];
                const float4 *T = s_tab + s_off[pos * P + l] - klo;
                df32 sr{0.f, 0.f}, si{0.f, 0.f};
                for (int k = klo; k <= khi; ++k) {
                    const float4 t = T[k];
                    const float4 v = s_x[k];
                    df_mac(sr, df32{t.x, t.y}, df32{v.x, v.y});
                    df_mac(sr, df32{-t.z, -t.w}, df32{v.z, v.w});
                    df_mac(si, df32{t.x, t.y}, df32{v.z, v.w});
                    df_mac(si, df32{t.z, t.w}, df32{v.x, v.y});
                }
                sr = df_norm(sr);
                si = df_norm(si);
                const double out_re = df_to_f64_scaled(sr, 0), out_im = df_to_f64_scaled(si, 0);
                double *xd = a.x + r * a.ldm + (int64_t)dst * 2 * P + 2 * l;
                if (UP) {
                    atomicAdd(xd, out_re);
                    atomicAdd(xd + 1, out_im);
                } else {
                    xd[0] = __ldcg(xd) + out_re;
                    xd[1] = __ldcg(xd + 1) + out_im;
                }
            }
            __syncwarp();   // s_x is rewritten for the next column
        }
        __threadfence();    // this box's results are visible before anything goes on from them
        __syncwarp();
        int next = -1;
        if (lane == 0) {
            if (UP) {       // the child that completes its parent's count goes on with the parent
                const int nd = a.need[par];
                if (nd > 0 && atomicAdd(a.ws + 2 + par, 1) == nd - 1) {
                    __threadfence();
                    next = par;
                }
            } else {        // on with the first child; the other three to the queue
                const int ch = a.child0[c];
                if (ch >= 0) {
                    const int s = atomicAdd(a.ws + 1, 3);
                    for (int k = 1; k < 4; ++k)
                        if (s + k - 1 < a.n_slots - a.n0) atomicExch(a.ws + 2 + a.n_boxes + s + k - 1, ch + k + 1);
                    next = ch;
                }
            }
        }
        c = __shfl_sync(0xffffffffu, next, 0);
        __threadfence();    // what the box's other writers made visible is seen before it is read
    }
}

// ------------------------------------------------------------------ host

// The complex form of four real 2P x 2P translation tables (rows 2l, 2l+1 and
// columns 2k, 2k+1 = Re, Im; block [[Re, -Im], [Im, Re]]) and every row's
// non-zero column range; false if a table is not of that form.
static bool complex_tables(const std::vector<double> &real4, int P, std::vector<double> &cplx,
                           std::vector<int16_t> &krange) {
    const int P2 = 2 * P;
    cplx.assign((size_t)4 * P * P * 2, 0.0);
    krange.assign((size_t)4 * P * 2, 0);
    for (int t = 0; t < 4; ++t)
        for (int l = 0; l < P; ++l) {
            int lo = P, hi = -1;
            for (int k = 0; k < P; ++k) {
                const double *T = &real4[(size_t)t * P2 * P2];
                const double re = T[(size_t)(2 * l) * P2 + 2 * k], im = T[(size_t)(2 * l + 1) * P2 + 2 * k];
                if (T[(size_t)(2 * l) * P2 + 2 * k + 1] != -im || T[(size_t)(2 * l + 1) * P2 + 2 * k + 1] != re)
                    return false;
                cplx[(((size_t)t * P + l) * P + k) * 2] = re;
                cplx[(((size_t)t * P + l) * P + k) * 2 + 1] = im;
                if (re != 0.0 || im != 0.0) {
                    lo = std::min(lo, k);
                    hi = std::max(hi, k);
                }
            }
            krange[((size_t)t * P + l) * 2] = (int16_t)(hi >= 0 ? lo : 0);
            krange[((size_t)t * P + l) * 2 + 1] = (int16_t)hi;
        }
    return true;
}


static int chain_nk(int P) {
    const int G = std::max(1, CH_THREADS / P);
    return (P + G - 1) / G <= 8 ? 8 : 16;
}

// Builds both chains of a plan:
// tables in the form's arithmetic, initially ready boxes, counts to wait for,
// and the zeroed queue block.  Leaves ChainPlan::ok false otherwise, and the
// per-level passes run the chains.
void setup_chains(vpx_plan *p, const std::vector<double> &m2m, const std::vector<double> &l2l) {
    ChainPlan &C = p->fmm.chain;
    C = ChainPlan();
    const int P = p->P, nb = (int)p->box_level.size();
    const bool mixed = p->opt.precision == VPX_PREC_MIXED;
    if (P > kMaxP || p->n_levels < 4) return;
    std::vector<double> cu, cd;
    std::vector<int16_t> ku, kd;
    if (!complex_tables(m2m, P, cu, ku) || !complex_tables(l2l, P, cd, kd)) return;
    auto upload_tab = [&](const std::vector<double> &c) -> void * {
        if (!mixed) return dev_upload(c);
        std::vector<float> f(c.size() * 2);
        for (size_t i = 0; i < c.size(); ++i) {
            const float hi = (float)c[i];
            f[2 * i] = hi;
            f[2 * i + 1] = (float)(c[i] - (double)hi);
        }
        return dev_upload(f);
    };
    C.tab_up = upload_tab(cu);
    C.tab_down = upload_tab(cd);
    C.kr_up = dev_upload(ku);
    C.kr_down = dev_upload(kd);
    std::vector<int32_t> need(nb, 0), up0, down0;
    int n_queued = 0;   // downward: the children queued (three of every non-leaf box at level >= 3)
    for (int b = 0; b < nb; ++b) {
        if (p->box_level[b] < 3) continue;
        if (p->box_level[b] == 3) down0.push_back(b);
        if (p->box_child0[b] >= 0) n_queued += 3;
        if (!p->box_nz[b]) continue;
        if (p->box_child0[b] < 0) {
            up0.push_back(b);
        } else {
            for (int k = 0; k < 4; ++k) need[b] += p->box_nz[p->box_child0[b] + k] ? 1 : 0;
        }
    }
    C.n0_up = (int)up0.size();
    C.n_up = C.n0_up;            // upward: the leaves are the only claims
    C.n0_down = (int)down0.size();
    C.n_down = C.n0_down + n_queued;
    std::vector<int32_t> up_of(2 * (size_t)nb, 0);
    for (int b = 0; b < nb; ++b) {
        const int pa = p->box_parent[b];
        up_of[2 * b] = pa;
        up_of[2 * b + 1] = pa >= 0 ? b - p->box_child0[pa] : 0;
    }
    C.up_of = dev_upload(up_of);
    C.items_up = dev_upload(up0);
    C.items_down = dev_upload(down0);
    C.need = dev_upload(need);
    C.ws_ints = (size_t)(2 + nb + C.n_up) + (size_t)(2 + nb + C.n_down);
    C.ws = dev_alloc<int>(C.ws_ints);
    if (mixed) {   // the warp-granular kernel's packed rows
        auto pack = [&](const std::vector<double> &c, const std::vector<int16_t> &kr, int &n) {
            std::vector<float> f;
            std::vector<int32_t> off(4 * (size_t)P);
            for (int t = 0; t < 4; ++t)
                for (int l = 0; l < P; ++l) {
                    off[(size_t)t * P + l] = (int32_t)(f.size() / 4);
                    for (int k = kr[((size_t)t * P + l) * 2]; k <= kr[((size_t)t * P + l) * 2 + 1]; ++k)
                        for (int ri = 0; ri < 2; ++ri) {
                            const double v = c[(((size_t)t * P + l) * P + k) * 2 + ri];
                            const float hi = (float)v;
                            f.push_back(hi);
                            f.push_back((float)(v - (double)hi));
                        }
                }
            n = (int)(f.size() / 4);
            return std::make_pair(dev_upload(f), dev_upload(off));
        };
        auto u = pack(cu, ku, C.np_up), d = pack(cd, kd, C.np_down);
        C.tabw_up = u.first;
        C.roff_up = u.second;
        C.tabw_down = d.first;
        C.roff_down = d.second;
        C.smem_w = (size_t)(std::max(C.np_up, C.np_down) + CW_WARPS * P) * 16 + (size_t)4 * P * 4 + (size_t)8 * P * 2;
        int occ_w = 0;
        VPX_CUDA(cudaFuncSetAttribute(k_wchain<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem_w));
        VPX_CUDA(cudaFuncSetAttribute(k_wchain<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem_w));
        VPX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_wchain<true>, CW_THREADS, C.smem_w));
        int dev = 0, nsm = 0;
        VPX_CUDA(cudaGetDevice(&dev));
        VPX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        C.max_ctas_w = std::max(1, std::min(occ_w, 4)) * nsm;
        if (occ_w <= 0) return;
    }
    int occ = 0;
    const int nk = chain_nk(P);
    if (mixed && nk == 8)
        VPX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chain<true, true, 8>, CH_THREADS, 0));
    else if (mixed)
        VPX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chain<true, true, 16>, CH_THREADS, 0));
    else if (nk == 8)
        VPX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chain<false, true, 8>, CH_THREADS, 0));
    else
        VPX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chain<false, true, 16>, CH_THREADS, 0));
    int dev = 0, nsm = 0;
    VPX_CUDA(cudaGetDevice(&dev));
    VPX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    C.max_ctas = std::max(1, std::min(occ, 8)) * nsm;
    C.ok = occ > 0;
}

void free_chains(vpx_plan *p) {
    ChainPlan &C = p->fmm.chain;
    dev_free(C.tab_up);
    dev_free(C.tab_down);
    dev_free(C.kr_up);
    dev_free(C.kr_down);
    dev_free(C.items_up);
    dev_free(C.items_down);
    dev_free(C.need);
    dev_free(C.up_of);
    dev_free(C.ws);
    dev_free(C.tabw_up);
    dev_free(C.tabw_down);
    dev_free(C.roff_up);
    dev_free(C.roff_down);
    C = ChainPlan();
}

// Zeroes both queue blocks (one memset, ahead of the upward chain).
void chain_reset(vpx_plan *p, cudaStream_t s) {
    const ChainPlan &C = p->fmm.chain;
    if (C.ok) VPX_CUDA(cudaMemsetAsync(C.ws, 0, C.ws_ints * sizeof(int), s));
}

// One launch of the upward (M2M) or downward (L2L) chain on the expansions x.
void chain_run(vpx_plan *p, bool up, double *x, int64_t ldm, int nrhs, cudaStream_t s) {
    const ChainPlan &C = p->fmm.chain;
    ChainArgs a;
    a.P = p->P;
    a.G = std::max(1, CH_THREADS / p->P);
    a.nrhs = nrhs;
    a.n_slots = up ? C.n_up : C.n_down;
    a.n0 = up ? C.n0_up : C.n0_down;
    if (a.n_slots == 0) return;
    a.ldm = ldm;
    a.items0 = up ? C.items_up : C.items_down;
    a.up_of = reinterpret_cast<const int2 *>(C.up_of);
    a.child0 = p->dt.box_child0;
    a.need = C.need;
    a.tab = up ? C.tab_up : C.tab_down;
    a.krange = up ? C.kr_up : C.kr_down;
    a.n_boxes = p->dt.n_boxes;
    a.ws = up ? C.ws : C.ws + (2 + p->dt.n_boxes + C.n_up);
    a.x = x;
    a.status = p->wk.status;
    const bool mixed = p->opt.precision == VPX_PREC_MIXED;
    if (mixed) {   // one warp per box
        WChainArgs w;
        w.P = a.P;
        w.nrhs = nrhs;
        w.n_slots = a.n_slots;
        w.n0 = a.n0;
        w.n_packed = up ? C.np_up : C.np_down;
        w.ldm = ldm;
        w.items0 = a.items0;
        w.up_of = a.up_of;
        w.child0 = a.child0;
        w.need = a.need;
        w.tabp = reinterpret_cast<const float4 *>(up ? C.tabw_up : C.tabw_down);
        w.roff = up ? C.roff_up : C.roff_down;
        w.krange = a.krange;
        w.ws = a.ws;
        w.n_boxes = a.n_boxes;
        w.x = x;
        w.status = a.status;
        const dim3 grid((unsigned)std::min((a.n_slots + CW_WARPS - 1) / CW_WARPS, C.max_ctas_w));
        if (up) launch_pdl(k_wchain<true>, grid, dim3(CW_THREADS), C.smem_w, s, w);
        else launch_pdl(k_wchain<false>, grid, dim3(CW_THREADS), C.smem_w, s, w);
        VPX_LAUNCH("k_wchain");
        return;
    }
    const dim3 grid((unsigned)std::min(a.n_slots, C.max_ctas));
    const size_t smem = 0;
    const int nk = chain_nk(p->P);
    if (nk == 8) {
        if (mixed && up) launch_pdl(k_chain<true, true, 8>, grid, dim3(CH_THREADS), smem, s, a);
        else if (mixed) launch_pdl(k_chain<true, false, 8>, grid, dim3(CH_THREADS), smem, s, a);
        else if (up) launch_pdl(k_chain<false, true, 8>, grid, dim3(CH_THREADS), smem, s, a);
        else launch_pdl(k_chain<false, false, 8>, grid, dim3(CH_THREADS), smem, s, a);
    } else {
        if (mixed && up) launch_pdl(k_chain<true, true, 16>, grid, dim3(CH_THREADS), smem, s, a);
        else if (mixed) launch_pdl(k_chain<true, false, 16>, grid, dim3(CH_THREADS), smem, s, a);
        else if (up) launch_pdl(k_chain<false, true, 16>, grid, dim3(CH_THREADS), smem, s, a);
        else launch_pdl(k_chain<false, false, 16>, grid, dim3(CH_THREADS), smem, s, a);
    }
    VPX_LAUNCH("k_chain");
}

}  // namespace vpx
