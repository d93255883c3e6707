// device_exec.cu -- the hot path: extension of f on cut leaves (Sections 3.2,
// 4.1) and the box FMM for the volume potential (eq. volinte) in FP64.
//
// Conventions (for every box B of side L at level l, centre c, half side h):
//   multipole  Phi(z) = a_0 log(z - c) + sum_{k>=1} at_k (L / (z - c))^k
//   local      Psi(z) = sum_{l>=0} bt_l ((z - c) / L)^l
//   V(x) = (1/2pi) Re Phi  (the complex log kernel; G = (1/2pi) log|x - y|).
// Leaf values are the K x K Gauss-Legendre node values of f^e on each leaf.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "dev_common.cuh"
#include "slice_math.cuh"
#include "ext.cuh"

namespace vpx {


__device__ inline double box_side_d(int level) { return ldexp(1.0, -level); }

// ---------------------------------------------------------------- extension

// regular leaves: copy data; exterior leaves outside every extension list: 0
// The leaf values that need no extension, one warp per leaf: a regular leaf
// takes the data at its nodes, an exterior leaf in no extension list is zero
// (cut leaves and extension-list leaves are the extension's).  In the mixed
// form (sl non-null) the warp also writes the leaf's exact bf16 slices and
// exponent, as the potential's passes read them (slice_math.cuh).
__global__ void __launch_bounds__(256) k_leafvals(int n_leaves, int KK, int kpad, const int32_t *leaf_cls,
                                                  const int32_t *owner_flag, const int64_t *reg_off, const double *f,
                                                  int64_t ldf, double *fe, int64_t ldfe, uint16_t *sl, int32_t *ex) {
    pdl_entry();
    const int rhs = blockIdx.y, lane = threadIdx.x & 31;
    const int leaf = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (leaf >= n_leaves) return;
    const int cls = leaf_cls[leaf];
    const bool reg = cls == kRegular;
    if (!reg && !(cls == kExterior && owner_flag[leaf] == 0)) return;
    double xv[kSliceMaxPerLane];
    uint64_t mb = 0;
    const double *src = reg ? f + rhs * ldf + reg_off[leaf] : nullptr;
    double *o = fe + rhs * ldfe + (int64_t)leaf * KK;
#pragma unroll
    for (int q = 0; q < kSliceMaxPerLane; ++q) {
        const int j = lane + 32 * q;
        xv[q] = (reg && j < KK) ? src[j] : 0.0;
        if (j < KK) o[j] = xv[q];
        const uint64_t t = slice_abs_bits(xv[q]);
        mb = t > mb ? t : mb;
    }
    if (!sl) return;
    const int e = slice_warp_expo(mb);
    uint16_t *out = sl + ((size_t)rhs * n_leaves + leaf) * kSlicesS * kpad;
#pragma unroll
    for (int q = 0; q < kSliceMaxPerLane; ++q) {
        const int j = lane + 32 * q;
        if (j >= kpad) break;
        uint16_t d[kSlicesS];
        slice_digits(slice_fixed_point(xv[q], e), d);
#pragma unroll
        for (int k = 0; k < kSlicesS; ++k) out[(size_t)k * kpad + j] = d[k];
    }
    if (lane == 0) ex[(size_t)rhs * n_leaves + leaf] = e;
}

// Extension along lines (Section 6.4): the value at each exterior grid point
// is the Floater-Hormann interpolant of the data at its eight line points,
// sum_q coef[q] f[src + q] with the coefficients from the host.  One thread
// per (exterior grid point, rhs).
__global__ void k_ext_rays(int n_ray, int Kb2, const int32_t *ray_c, const int32_t *ray_g, const int64_t *ray_src,
                           const double *ray_coef, const double *f, int64_t ldf, double *F, int64_t ldF) {
    pdl_entry();
    const int k = blockIdx.x * blockDim.x + threadIdx.x, rhs = blockIdx.y;
    if (k >= n_ray) return;
    const double *fr = f + rhs * ldf + ray_src[k];
    const double *cf = ray_coef + (size_t)k * 8;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += cf[q] * fr[q];
    F[rhs * ldF + (int64_t)ray_c[k] * Kb2 + ray_g[k]] = s;
}

// One block per (cut leaf, rhs).  c = A_I^+ f_I; the Kbar x Kbar Chebyshev grid
// on Sbar takes the data at interior nodes and A_{Xbar^E,G} c at exterior
// nodes; its Chebyshev coefficients truncated to m + n < Kbar (eq.
// chebexpbarS) are evaluated at the cut leaf's exterior nodes and at all nodes
// of the exterior leaves in its extension list.
__global__ void k_extend(ExtArgs a) {
    pdl_entry();
    extern __shared__ double sm[];
    const int c = blockIdx.x, rhs = blockIdx.y;
    const int K = a.K, KK = K * K, Kb = a.Kbar, Kb2 = Kb * Kb, NG = a.NG;
    const int nI = a.n_interior[c];
    double *fI = sm;                 // nI
    double *cc = fI + nI;            // NG
    double *F = cc + NG;             // Kb2   grid values, index by*Kb + ax
    double *T1 = F + Kb2;            // Kb2
    double *al = T1 + Kb2;           // Kb2   alpha[m*Kb + n]
    double *Tx = al + Kb2;           // K*Kb  T_m at the target x nodes
    double *Ty = Tx + K * Kb;        // K*Kb
    double *G = Ty + K * Kb;         // Kb*K
    const double *f = a.f + rhs * a.ldf + a.stencil_off[c];
    for (int i = threadIdx.x; i < nI; i += blockDim.x) fI[i] = f[i];
    __syncthreads();
    // c = P_S f_I : one warp per row (universal stencil only)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const double *P = a.ray_F ? nullptr : a.pinv + a.pinv_off[c];
    for (int k = warp; !a.ray_F && k < NG; k += nwarp) {
        double s = 0.0;
        for (int i = lane; i < nI; i += 32) s += P[(size_t)k * nI + i] * fI[i];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) cc[k] = s;
    }
    __syncthreads();
    const int32_t *gs = a.grid_src + (size_t)c * Kb2;
    for (int g = threadIdx.x; g < Kb2; g += blockDim.x) {
        int src = gs[g];
        if (src >= 0) {
            F[g] = fI[src];
        } else if (a.ray_F) {
            F[g] = a.ray_F[rhs * a.ldR + (int64_t)c * Kb2 + g];
        } else {
            double s = 0.0;
            const double *Ar = a.A_grid + (size_t)g * NG;
            for (int k = 0; k < NG; ++k) s += Ar[k] * cc[k];
            F[g] = s;
        }
    }
    __syncthreads();
    // T1[m][by] = sum_ax C[m][ax] F[by][ax];  alpha[m][n] = sum_by T1[m][by] C[n][by]
    for (int e = threadIdx.x; e < Kb2; e += blockDim.x) {
        int m = e / Kb, by = e % Kb;
        double s = 0.0;
        for (int ax = 0; ax < Kb; ++ax) s += a.cheb_inv[m * Kb + ax] * F[by * Kb + ax];
        T1[m * Kb + by] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Kb2; e += blockDim.x) {
        int m = e / Kb, n = e % Kb;
        double s = 0.0;
        if (m + n < Kb)
            for (int by = 0; by < Kb; ++by) s += T1[m * Kb + by] * a.cheb_inv[n * Kb + by];
        al[m * Kb + n] = s;
    }
    __syncthreads();
    const int leaf = a.cut_leaf[c];
    const int ls = a.leaf_level[leaf];
    const double sS = box_side_d(ls);
    const double cxS = -0.5 + (a.leaf_ix[leaf] + 0.5) * sS, cyS = -0.5 + (a.leaf_iy[leaf] + 0.5) * sS;
    const double r = 1.5 * sS;   // half side of Sbar
    const int nown = a.owned_off[c + 1] - a.owned_off[c];
    for (int tgt = -1; tgt < nown; ++tgt) {
        const int tl = (tgt < 0) ? leaf : a.owned[a.owned_off[c] + tgt];
        const double sT = box_side_d(a.leaf_level[tl]);
        const double cxT = -0.5 + (a.leaf_ix[tl] + 0.5) * sT, cyT = -0.5 + (a.leaf_iy[tl] + 0.5) * sT;
        for (int e = threadIdx.x; e < 2 * K; e += blockDim.x) {
            int i = e % K;
            double z = (e < K) ? (cxT - cxS + 0.5 * sT * a.tnodes[i]) / r : (cyT - cyS + 0.5 * sT * a.tnodes[i]) / r;
            double *T = (e < K) ? Tx + i * Kb : Ty + i * Kb;
            T[0] = 1.0;
            if (Kb > 1) T[1] = z;
            for (int m = 2; m < Kb; ++m) T[m] = 2.0 * z * T[m - 1] - T[m - 2];
        }
        __syncthreads();
        // G[n][ax] = sum_m alpha[m][n] Tx[ax][m]
        for (int e = threadIdx.x; e < Kb * K; e += blockDim.x) {
            int n = e / K, ax = e % K;
            double s = 0.0;
            for (int m = 0; m + n < Kb; ++m) s += al[m * Kb + n] * Tx[ax * Kb + m];
            G[n * K + ax] = s;
        }
        __syncthreads();
        double *out = a.fe + rhs * a.ldfe + (int64_t)tl * KK;
        const int32_t *ns = a.node_src + (size_t)c * KK;
        for (int j = threadIdx.x; j < KK; j += blockDim.x) {
            int ax = j % K, by = j / K;
            if (tgt < 0 && ns[j] >= 0) {
                out[j] = fI[ns[j]];
            } else {
                double s = 0.0;
                for (int n = 0; n < Kb; ++n) s += Ty[by * Kb + n] * G[n * K + ax];
                out[j] = s;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- boundary

// The last launch of the potential: blocks [0, nan_blocks) check V for
// non-finite values (status VPX_ERR_NAN); the rest interpolate V at the
// boundary nodes, one warp per node: V(x) = sum_b w_y[b] sum_a w_x[a] V_leaf[b][a].
__global__ void k_finish(int64_t n_v, int nan_blocks, int nb, int K, const int32_t *bleaf, const double *bw,
                         const double *v, int64_t ldv, double *vb, int64_t ldb, int *status) {
    pdl_entry();
    const int rhs = blockIdx.y;
    if ((int)blockIdx.x < nan_blocks) {   // grid-stride over the leaf values
        bool bad = false;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_v; i += (int64_t)nan_blocks * blockDim.x)
            bad |= !isfinite(v[rhs * ldv + i]);
        if (bad) set_status(status, VPX_ERR_NAN);
        return;
    }
    const int k = (blockIdx.x - nan_blocks) * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= nb || vb == nullptr) return;
    const double *w = bw + (size_t)k * 2 * K;
    const double *V = v + rhs * ldv + (int64_t)bleaf[k] * K * K;
    constexpr int kMaxPerLane = kMaxK * kMaxK / 32;
    double vv[kMaxPerLane], wx[kMaxPerLane], wy[kMaxPerLane];
#pragma unroll
    for (int q = 0; q < kMaxPerLane; ++q) {
        const int j = lane + 32 * q;
        const bool in = j < K * K;
        vv[q] = in ? V[j] : 0.0;
        wx[q] = in ? w[j % K] : 0.0;
        wy[q] = in ? w[K + j / K] : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxPerLane; ++q) s += wy[q] * wx[q] * vv[q];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) vb[rhs * ldb + k] = s;
}

// Net charge A^e = \iint f^e (Section 6.2), by each leaf's tensor
// Gauss-Legendre rule: sum_leaves (side/2)^2 sum_j w2[j] f^e[leaf][j].  The
// first kernel gives each block a fixed set of leaves (one warp per leaf,
// leaves strided by the grid) and writes the block's sum; the second adds the
// block sums of a right-hand side in a fixed order, so the result does not
// depend on scheduling.  The grid size depends on n_leaves only.
__global__ void __launch_bounds__(256) k_charge_partial(int n_leaves, int KK, const int32_t *leaf_level,
                                                        const double *w2, const double *fe, int64_t ldfe,
                                                        double *part) {
    pdl_entry();
    const int rhs = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double *F = fe + rhs * ldfe;
    double s = 0.0;
    for (int i = blockIdx.x * nw + warp; i < n_leaves; i += gridDim.x * nw) {
        double t = 0.0;
        for (int j = lane; j < KK; j += 32) t += w2[j] * F[(int64_t)i * KK + j];
        const double h = ldexp(0.5, -leaf_level[i]);
        s += t * h * h;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    if (lane == 0) ws[warp] = s;
    __syncthreads();
    if (warp == 0) {
        s = lane < nw ? ws[lane] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[(int64_t)rhs * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_charge_final(int nparts, const double *part, double *charge) {
    pdl_entry();
    const int rhs = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += part[(int64_t)rhs * nparts + k];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    if (lane == 0) ws[warp] = s;
    __syncthreads();
    if (warp == 0) {
        s = lane < 8 ? ws[lane] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) charge[rhs] = s;
    }
}

// ------------------------------------------------------------ host side

// Dynamic shared memory of the extension kernels (8-byte words: FP64 or a
// double-float pair) for the largest cut leaf.
static size_t extension_smem(const vpx_plan *p) {
    const StencilInfo &st = p->st;
    int maxI = 0;
    for (int c = 0; c < (int)st.cut_leaf.size(); ++c) maxI = std::max(maxI, st.n_interior[c]);
    return sizeof(double) * ((size_t)maxI + st.NG + 3 * st.Kbar * st.Kbar + 3 * p->K * st.Kbar);
}

// Opt the extension kernels into the dynamic shared memory they need.
static void prepare_extension(vpx_plan *p) {
    const size_t smem = extension_smem(p);
    if (smem > 48 * 1024) VPX_CUDA(cudaFuncSetAttribute(k_extend, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the coefficient kernel runs for the universal stencil only (its shared
    // memory holds a cut leaf's interior stencil values, which along lines
    // would be the line points as well)
    if (p->opt.precision == VPX_PREC_MIXED)
        extend_df_prepare(p->ext.mode == 1 ? 0 : p->ext.max_interior, p->K, p->st.Kbar);
}

// Per-plan index arrays of the execute path: non-zero leaves and the
// extension-list membership flag of every leaf.
void setup_near_pairs(vpx_plan *p) {
    const int nl = (int)p->tree.leaves.size();
    std::vector<int32_t> nz, of(nl, 0);
    for (int i = 0; i < nl; ++i) {
        if (p->leaf_nz[i]) nz.push_back(i);
        of[i] = p->tree.leaves[i].owner >= 0 ? 1 : 0;
    }
    p->wk.nz_leaves = dev_upload(nz);
    p->wk.n_nz_leaves = (int)nz.size();
    p->ext.owned_flag_dev = dev_upload(of);
    prepare_extension(p);
}

void ev_record(vpx_plan *p, int i, cudaStream_t s) {
    if (!p->timing) return;
    if (!p->events[i]) VPX_CUDA(cudaEventCreate((cudaEvent_t *)&p->events[i]));
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->events[i], s));
}

void ev_record_pass(vpx_plan *p, int i, cudaStream_t s) { ev_record(p, i, s); }

// Leaf values f^e of every leaf into fe; with slice = true (mixed form) also
// their exact slices into the plan's slice buffer, written by the kernels that
// produce the values, so that the potential need not slice them again.
static void run_extension(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *fe, int64_t ldfe,
                          cudaStream_t s, bool slice = false) {
    const int nl = p->dt.n_leaves, KK = p->KK;
    const int64_t n = (int64_t)nl * KK;
    const int kpad_f = (KK + 31) / 32 * 32;
    uint16_t *sl = slice ? p->fmm.fe_sl : nullptr;
    int32_t *ex = slice ? p->fmm.fe_ex : nullptr;
    // regular and unowned exterior leaves on the second stream, beside the
    // extension (which writes only the cut leaves and their extension lists)
    cudaStream_t aux = (cudaStream_t)p->aux_stream;
    if (n > 0) {
        VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_lvf, s));
        VPX_CUDA(cudaStreamWaitEvent(aux, (cudaEvent_t)p->ev_lvf, 0));
        dim3 g((unsigned)((nl + 7) / 8), nrhs);
        launch_pdl(k_leafvals, g, dim3(256), 0, aux, nl, KK, kpad_f, p->dt.leaf_cls, p->ext.owned_flag_dev,
                   p->ext.reg_leaf_off, f, ldf, fe, ldfe, sl, ex);
        VPX_LAUNCH("k_leafvals");
        VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_lv, aux));
    }
    if (p->ext.ncut > 0) {
        const StencilInfo &st = p->st;
        ExtArgs a;
        a.K = p->K;
        a.Kbar = st.Kbar;
        a.NG = st.NG;
        a.cut_leaf = p->ext.cut_leaf;
        a.n_interior = p->ext.n_interior;
        a.grid_src = p->ext.grid_src;
        a.node_src = p->ext.node_src;
        a.owned_off = p->ext.owned_off;
        a.owned = p->ext.owned;
        a.stencil_off = p->ext.stencil_off;
        a.pinv_off = p->ext.pinv_off;
        a.pinv = p->ext.pinv;
        a.A_grid = p->ext.A_grid;
        a.cheb_inv = p->ext.cheb_inv;
        a.tnodes = p->tab.tnodes;
        a.leaf_level = p->ext.leaf_level;
        a.leaf_ix = p->ext.leaf_ix;
        a.leaf_iy = p->ext.leaf_iy;
        a.f = f;
        a.ldf = ldf;
        a.fe = fe;
        a.ldfe = ldfe;
        a.pinv_df = reinterpret_cast<const float2 *>(p->ext.pinv_df);
        a.cheb_df = reinterpret_cast<const float2 *>(p->ext.cheb_df);
        a.fe_sl = sl;
        a.fe_ex = ex;
        a.n_leaves = nl;
        a.kpad = kpad_f;
        const size_t smem = extension_smem(p);
        DevExt &xe = p->ext;
        const int Kb2e = p->st.Kbar * p->st.Kbar;
        const int64_t ldFe = (int64_t)xe.ncut * Kb2e;
        if (xe.mode == 1 && xe.n_ray > 0) {   // exterior grid values along lines
            launch_pdl(k_ext_rays, dim3((unsigned)((xe.n_ray + 255) / 256), nrhs), dim3(256), 0, s, xe.n_ray, Kb2e,
                       (const int32_t *)xe.ray_c, (const int32_t *)xe.ray_g, (const int64_t *)xe.ray_src,
                       (const double *)xe.ray_coef, f, ldf, xe.Fall, ldFe);
            VPX_LAUNCH("k_ext_rays");
        }
        if (xe.mode == 1 && p->opt.precision == VPX_PREC_MIXED) {
            launch_ext_eval_df(a, xe.ncut, xe.n_tgt, xe.tgt_cut, xe.tgt_leaf,
                               reinterpret_cast<const ExtTgtGeo *>(xe.tgt_geo), xe.Fall, ldFe,
                               reinterpret_cast<float2 *>(xe.alpha), nrhs, p->wk.status, s);
        } else if (xe.mode == 1) {
            a.ray_F = xe.Fall;
            a.ldR = ldFe;
            launch_pdl(k_extend, dim3(p->ext.ncut, nrhs), dim3(256), smem, s, a);
            VPX_LAUNCH("k_extend");
        } else if (p->opt.precision == VPX_PREC_MIXED) {
            DevExt &x = p->ext;
            a.pinv_df_off = x.pinv_df_off;
            const int Kb2 = p->st.Kbar * p->st.Kbar;
            const int64_t ldc = (int64_t)x.ncut * p->st.NG, ldF = (int64_t)x.ncut * Kb2;
            launch_ext_coeff_df(a, x.ncut, x.max_interior, nrhs, x.cbuf, ldc, p->wk.status, s);
            VecSet vc{x.cbuf, ldc, p->st.NG, nullptr, nullptr, x.ncut, 0};
            gemm_run(x.grid_pass, vc, x.Fall, ldF, nrhs, true, s);
            launch_ext_eval_df(a, x.ncut, x.n_tgt, x.tgt_cut, x.tgt_leaf,
                               reinterpret_cast<const ExtTgtGeo *>(x.tgt_geo), x.Fall, ldF,
                               reinterpret_cast<float2 *>(x.alpha), nrhs, p->wk.status, s);
        } else {
            launch_pdl(k_extend, dim3(p->ext.ncut, nrhs), dim3(256), smem, s, a);
            VPX_LAUNCH("k_extend");
        }
    }
    if (n > 0) VPX_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)p->ev_lv, 0));
}

void run_potential_passes(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                          int64_t ldb, double *mp, double *lo, cudaStream_t s, bool fe_sliced);

// The box FMM and the boundary interpolation, with the multipole and local
// expansions in the scratch arrays mp and lo (each nrhs x n_boxes x 2P doubles);
// fe_sliced: the leaf values' slices are already in the plan's slice buffer.
void run_potential_scratch(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                           int64_t ldb, double *mp, double *lo, cudaStream_t s, bool fe_sliced) {
    run_potential_passes(p, fe, ldfe, nrhs, v, ldv, vb, ldb, mp, lo, s, fe_sliced);
    const int nbd = (vb != nullptr) ? (int)p->bdry_leaf.size() : 0;
    const int64_t n_v = (int64_t)p->dt.n_leaves * p->KK;
    // a few thousand values per block: a block per 256 values spent most of
    // the kernel's time starting blocks
    const int nan_blocks = (int)std::min<int64_t>((n_v + 2047) / 2048, 1024);
    const int blocks = nan_blocks + (nbd + 7) / 8;
    if (blocks > 0) {
        launch_pdl(k_finish, dim3(blocks, nrhs), dim3(256), 0, s, n_v, nan_blocks, nbd, p->K, p->wk.bdry_leaf, p->wk.bdry_w, v, ldv,
                                                    vb, ldb, p->wk.status);
        VPX_LAUNCH("k_finish");
    }
    ev_record(p, 8, s);
}

static void run_potential(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                          int64_t ldb, cudaStream_t s) {
    run_potential_scratch(p, fe, ldfe, nrhs, v, ldv, vb, ldb, p->wk.mpole, p->wk.local, s, false);
}

void device_extend(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *fe, int64_t ldfe, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = stream;
    run_extension(p, f, nrhs, ldf, fe, ldfe, s);
}

void device_potential(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                      int64_t ldb, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = stream;
    ev_record(p, 0, s);
    run_potential(p, fe, ldfe, nrhs, v, ldv, vb, ldb, s);
}

void device_net_charge(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *charge, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = stream;
    const int nparts = charge_blocks(p->dt.n_leaves);
    launch_pdl(k_charge_partial, dim3(nparts, nrhs), dim3(256), 0, s, p->dt.n_leaves, p->KK,
               (const int32_t *)p->ext.leaf_level, (const double *)p->tab.w2, fe, ldfe, p->wk.charge_part);
    VPX_LAUNCH("k_charge_partial");
    launch_pdl(k_charge_final, dim3(nrhs), dim3(256), 0, s, nparts, (const double *)p->wk.charge_part, charge);
    VPX_LAUNCH("k_charge_final");
}

static void execute_sequence(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *v, int64_t ldv, double *vb,
                             int64_t ldb, cudaStream_t s) {
    const int64_t ldfe = (int64_t)p->dt.n_leaves * p->KK;
    const bool mixed = p->opt.precision == VPX_PREC_MIXED;
    ev_record(p, 0, s);
    run_extension(p, f, nrhs, ldf, p->wk.fe, ldfe, s, mixed);
    run_potential_scratch(p, p->wk.fe, ldfe, nrhs, v, ldv, vb, ldb, p->wk.mpole, p->wk.local, s, mixed);
}

// The whole sequence (about 25 kernels) is captured into a CUDA graph on the
// first call with a given set of buffers, strides and nrhs, and replayed on
// later calls; calls on the legacy default stream run the launches directly.
void device_execute(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *v, int64_t ldv, double *vb,
                    int64_t ldb, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = stream;
    static const bool no_graph = getenv("VPX_NO_GRAPH") != nullptr;
    if (s == nullptr || no_graph || p->timing) {   // per-pass timing runs the launches directly
        execute_sequence(p, f, nrhs, ldf, v, ldv, vb, ldb, s);
        return;
    }
    const int64_t key[10] = {(int64_t)(uintptr_t)f, ldf, (int64_t)(uintptr_t)v, ldv, (int64_t)(uintptr_t)vb, ldb,
                             nrhs, p->timing ? 1 : 0, (int64_t)(uintptr_t)s, p->tune_epoch};
    bool hit = p->graph_exec != nullptr;
    for (int i = 0; i < 10 && hit; ++i) hit = key[i] == p->graph_key[i];
    if (!hit) {
        if (p->graph_exec) {
            cudaGraphExecDestroy((cudaGraphExec_t)p->graph_exec);
            p->graph_exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        VPX_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            execute_sequence(p, f, nrhs, ldf, v, ldv, vb, ldb, s);
        } catch (...) {
            cudaStreamEndCapture(s, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        VPX_CUDA(cudaStreamEndCapture(s, &graph));
        size_t n_nodes = 0;
        VPX_CUDA(cudaGraphGetNodes(graph, nullptr, &n_nodes));
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if (n_nodes) VPX_CUDA(cudaGraphGetNodes(graph, nodes.data(), &n_nodes));
        int64_t nk = 0;
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            VPX_CUDA(cudaGraphNodeGetType(nd, &t));
            if (t == cudaGraphNodeTypeKernel) ++nk;
        }
        p->graph_kernels = nk;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        VPX_CUDA(e);
        p->graph_exec = exec;
        for (int i = 0; i < 10; ++i) p->graph_key[i] = key[i];
    }
    VPX_CUDA(cudaGraphLaunch((cudaGraphExec_t)p->graph_exec, s));
}

// A batch of plans in one graph.  One cached graph per process (the last
// batch key); the key holds every plan's unique id, so a destroyed plan whose
// address is reused never matches.
static std::mutex g_batch_mu;
static std::vector<int64_t> g_batch_key;
static cudaGraphExec_t g_batch_exec = nullptr;

void device_execute_batch(int n, vpx_plan *const *plans, const double *const *f, const int *nrhs, const int64_t *ldf,
                          double *const *v, const int64_t *ldv, double *const *vb, const int64_t *ldb, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    bool direct = s == nullptr || getenv("VPX_NO_GRAPH") != nullptr;
    for (int i = 0; i < n; ++i) direct = direct || plans[i]->timing;
    if (direct) {
        for (int i = 0; i < n; ++i) {
            plans[i]->last_stream = stream;
            execute_sequence(plans[i], f[i], nrhs[i], ldf[i], v[i], ldv[i], vb[i], ldb[i], s);
        }
        return;
    }
    std::vector<int64_t> key = {n, (int64_t)(uintptr_t)s};
    for (int i = 0; i < n; ++i) {
        const int64_t k[9] = {(int64_t)plans[i]->uid, plans[i]->tune_epoch, (int64_t)(uintptr_t)f[i], nrhs[i],
                              ldf[i], (int64_t)(uintptr_t)v[i], ldv[i], (int64_t)(uintptr_t)vb[i], ldb[i]};
        key.insert(key.end(), k, k + 9);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    if (key != g_batch_key || !g_batch_exec) {
        if (g_batch_exec) {
            cudaGraphExecDestroy(g_batch_exec);
            g_batch_exec = nullptr;
        }
        g_batch_key.clear();
        cudaGraph_t graph = nullptr;
        VPX_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            // every tree forks from one point of `stream` and joins back at the
            // end, so the trees' passes are independent branches of the graph
            VPX_CUDA(cudaEventRecord((cudaEvent_t)plans[0]->ev_bfork, s));
            for (int i = 0; i < n; ++i) {
                vpx_plan *p = plans[i];
                cudaStream_t ps = (cudaStream_t)p->stream;
                VPX_CUDA(cudaStreamWaitEvent(ps, (cudaEvent_t)plans[0]->ev_bfork, 0));
                execute_sequence(p, f[i], nrhs[i], ldf[i], v[i], ldv[i], vb[i], ldb[i], ps);
                VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_bjoin, ps));
            }
            for (int i = 0; i < n; ++i) VPX_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)plans[i]->ev_bjoin, 0));
        } catch (...) {
            cudaStreamEndCapture(s, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        VPX_CUDA(cudaStreamEndCapture(s, &graph));
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        VPX_CUDA(e);
        g_batch_exec = exec;
        g_batch_key = key;
    }
    VPX_CUDA(cudaGraphLaunch(g_batch_exec, s));
    for (int i = 0; i < n; ++i) plans[i]->last_stream = stream;
}

// ------------------------------------------------------------------ autotuner
//
// The mixed-form passes that two engines or two tile widths can run (the near
// field on tcgen05 or mma.sync; 8 or 32 pairs per mma.sync tile) are tuned on
// the plans' own data.  One execute per plan records every pass call; each
// candidate then replays the call into scratch memory and must agree with the
// default choice to 1e-12 of the maximum (the candidates differ only in how
// the exact order sums are split).  The choice is made by timing the whole
// step -- the captured graph of the plan, or of the batch -- because a pass
// timed alone favours wide tiles (fewer table reads), while inside the step
// it shares the GPU with the passes on the other streams.  One sweep of
// coordinate descent over the pass roles (the same member of every plan:
// near field, M2L, ...) keeps, role by role, the candidate with the shortest
// step if it beats the current choice by 3 %.  Single-plan results are cached
// per pass-shape signature.

bool gemm_frag_eligible(const GemmPass &g, const VecSet &vs);
bool gemm_ws_eligible(const GemmPass &g, const VecSet &vs);

static std::mutex g_tune_mu;
static std::map<std::vector<int64_t>, std::vector<GemmChoice>> g_tune_cache;

static void shape_key(const GemmCall &c, std::vector<int64_t> &key) {
    const GemmPass &g = *c.g;
    int64_t lg = 0;
    while ((int64_t(1) << lg) < (int64_t)g.n_pairs) ++lg;
    const int64_t k[10] = {g.M, g.Kd, g.Kpad, g.ntab, (int64_t)kSlicesS, lg, c.nrhs, c.vs.slices != nullptr ? 1 : 0,
                           gemm_ws_eligible(g, c.vs) ? 1 : 0, g.add};
    key.insert(key.end(), k, k + 10);
}

// elements from `out` that one call may write: (nrhs - 1) ldo + max dst + M
static int64_t call_footprint(const GemmCall &c) {
    int64_t mx = 0;
    for (const GPair &q : c.g->h_pairs) mx = std::max<int64_t>(mx, q.dst);
    return (int64_t)(c.nrhs - 1) * c.ldo + mx + c.g->M;
}

struct TunePass {
    GemmCall call;
    size_t role;                      // byte offset of the pass inside its plan
    GemmChoice dflt;
    std::vector<GemmChoice> cand;     // candidates that agree with the default
};

// np_f 0 means "any width": the tcgen05 engine does not use the fragment tiles
static bool same_choice(GemmChoice a, GemmChoice b) {
    return a.engine == b.engine && (a.np_f == b.np_f || a.np_f == 0 || b.np_f == 0);
}

void device_autotune(int n, vpx_plan *const *plans, const double *const *f, const int *nrhs, const int64_t *ldf,
                     void *stream, int *n_passes, int *n_changed) {
    cudaStream_t s = (cudaStream_t)stream;
    int tuned = 0, changed = 0;
    bool any_mixed = false;
    for (int i = 0; i < n; ++i) any_mixed = any_mixed || plans[i]->opt.precision == VPX_PREC_MIXED;
    if (!any_mixed) {
        if (n_passes) *n_passes = 0;
        if (n_changed) *n_changed = 0;
        return;
    }
    std::vector<double *> v(n, nullptr), vb(n, nullptr);
    std::vector<int64_t> ldv(n), ldb(n);
    double *scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release = [&] {
        gemm_set_recorder(nullptr);
        dev_free(scratch);
        for (int i = 0; i < n; ++i) {
            dev_free(v[i]);
            dev_free(vb[i]);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    std::vector<TunePass> tp;
    try {
        // 1. record the pass calls of every plan (one execute each)
        for (int i = 0; i < n; ++i) {
            vpx_plan *p = plans[i];
            ldv[i] = std::max<int64_t>((int64_t)p->dt.n_leaves * p->KK, 1);
            ldb[i] = std::max<int64_t>((int64_t)p->bdry_xy.size() / 2, 1);
            v[i] = dev_alloc<double>((size_t)ldv[i] * nrhs[i]);
            vb[i] = p->bdry_xy.empty() ? nullptr : dev_alloc<double>((size_t)ldb[i] * nrhs[i]);
            if (p->opt.precision != VPX_PREC_MIXED) continue;
            std::vector<GemmCall> calls;
            gemm_set_recorder(&calls);
            execute_sequence(p, f[i], nrhs[i], ldf[i], v[i], ldv[i], vb[i], ldb[i], s);
            gemm_set_recorder(nullptr);
            std::vector<const GemmPass *> seen;
            for (const GemmCall &c : calls) {
                if (std::find(seen.begin(), seen.end(), c.g) != seen.end()) continue;   // first call of a pass
                seen.push_back(c.g);
                if (!gemm_frag_eligible(*c.g, c.vs)) continue;
                const size_t role = (size_t)((const char *)c.g - (const char *)p);
                if (role >= sizeof(vpx_plan)) continue;
                TunePass t{c, role, gemm_choice(*c.g), {}};
                // engine 0 routes to tcgen05 where eligible, else to the fragment engine;
                // engine 1 forces the fragment engine (a distinct choice only where tcgen05 is
                // eligible; elsewhere both values mean the fragment engine, so the pass keeps its own)
                const bool tc = gemm_ws_eligible(*c.g, c.vs);
                const int frag_engine = tc ? 1 : c.g->engine;
                if (tc) t.cand.push_back(GemmChoice{0, 0});
                t.cand.push_back(GemmChoice{frag_engine, 8});
                t.cand.push_back(GemmChoice{frag_engine, 32});
                bool has_default = false;
                for (const GemmChoice &x : t.cand) has_default = has_default || same_choice(x, t.dflt);
                if (!has_default) fail(VPX_ERR_STATE, "autotune: the default choice is not a candidate");
                tp.push_back(t);
            }
        }
        VPX_CUDA(cudaStreamSynchronize(s));
        // 2. every candidate must reproduce the default choice's output
        int64_t fp = 1;
        for (const TunePass &t : tp) fp = std::max(fp, call_footprint(t.call));
        scratch = dev_alloc<double>((size_t)fp);
        std::vector<double> ref, got;
        for (TunePass &t : tp) {
            GemmPass &g = *t.call.g;
            const size_t m = (size_t)call_footprint(t.call);
            for (int pass = 0; pass < 2; ++pass) {   // pass 0: the default, pass 1: the others
                for (const GemmChoice &c : t.cand) {
                    if (same_choice(c, t.dflt) != (pass == 0)) continue;
                    gemm_set_choice(g, c);
                    VPX_CUDA(cudaMemsetAsync(scratch, 0, m * sizeof(double), s));
                    gemm_run(g, t.call.vs, scratch, t.call.ldo, t.call.nrhs, true, s);
                    got.resize(m);
                    VPX_CUDA(cudaMemcpyAsync(got.data(), scratch, m * sizeof(double), cudaMemcpyDeviceToHost, s));
                    VPX_CUDA(cudaStreamSynchronize(s));
                    if (pass == 0) {
                        ref = got;
                        continue;
                    }
                    if (ref.size() != m) fail(VPX_ERR_STATE, "autotune: no reference output for a pass");
                    double mx = 0.0, d = 0.0;
                    for (size_t i = 0; i < m; ++i) {
                        mx = std::max(mx, std::fabs(ref[i]));
                        d = std::max(d, std::fabs(got[i] - ref[i]));
                    }
                    if (!(d <= 1e-12 * mx)) {
                        gemm_set_choice(g, t.dflt);
                        fail(VPX_ERR_STATE, "autotune: an engine variant disagrees with the default");
                    }
                }
            }
            gemm_set_choice(g, t.dflt);
        }
        dev_free(scratch);
        // 3. roles in call order; candidates common to every pass of a role
        std::vector<size_t> roles;
        for (const TunePass &t : tp)
            if (std::find(roles.begin(), roles.end(), t.role) == roles.end()) roles.push_back(t.role);
        std::vector<int64_t> sig;
        if (n == 1) {
            for (const TunePass &t : tp) shape_key(t.call, sig);
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tune_cache.find(sig);
            if (it != g_tune_cache.end() && it->second.size() == tp.size()) {
                for (size_t k = 0; k < tp.size(); ++k) {
                    gemm_set_choice(*tp[k].call.g, it->second[k]);
                    changed += !same_choice(it->second[k], tp[k].dflt);
                }
                tuned = (int)tp.size();
                sig.clear();
                roles.clear();   // nothing left to time
            }
        }
        // 4. coordinate descent on the time of the whole step
        VPX_CUDA(cudaEventCreate(&e0));
        VPX_CUDA(cudaEventCreate(&e1));
        auto step = [&] {
            if (n == 1) device_execute(plans[0], f[0], nrhs[0], ldf[0], v[0], ldv[0], vb[0], ldb[0], s);
            else device_execute_batch(n, plans, f, nrhs, ldf, v.data(), ldv.data(), vb.data(), ldb.data(), s);
        };
        auto step_ms = [&] {
            for (int i = 0; i < n; ++i) ++plans[i]->tune_epoch;   // recapture with the current choices
            step();
            step();
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                VPX_CUDA(cudaEventRecord(e0, s));
                for (int r = 0; r < 5; ++r) step();
                VPX_CUDA(cudaEventRecord(e1, s));
                VPX_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                VPX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                best = std::min(best, ms);
            }
            return best;
        };
        for (size_t role : roles) {
            std::vector<GemmChoice> common;
            bool first = true;
            for (const TunePass &t : tp) {
                if (t.role != role) continue;
                if (first) {
                    common = t.cand;
                    first = false;
                    continue;
                }
                std::vector<GemmChoice> keep;
                for (const GemmChoice &c : common)
                    for (const GemmChoice &d : t.cand)
                        if (same_choice(c, d)) keep.push_back(c);
                common = keep;
            }
            // the current choices first; another wins only by 3 % (replay-to-replay noise is ~1-2 %)
            std::vector<std::pair<TunePass *, GemmChoice>> current;
            for (TunePass &t : tp)
                if (t.role == role) current.push_back({&t, gemm_choice(*t.call.g)});
            const float cur_ms = step_ms();
            float best_ms = cur_ms;
            GemmChoice best{-1, 0};
            for (const GemmChoice &c : common) {
                for (TunePass &t : tp)
                    if (t.role == role) gemm_set_choice(*t.call.g, c);
                const float ms = step_ms();
                if (ms < 0.97f * cur_ms && ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            for (auto &pc : current) gemm_set_choice(*pc.first->call.g, best.engine >= 0 ? best : pc.second);
        }
        if (!roles.empty()) {
            std::vector<GemmChoice> chosen;
            for (const TunePass &t : tp) {
                const GemmChoice c = gemm_choice(*t.call.g);
                chosen.push_back(c);
                changed += !same_choice(c, t.dflt);
            }
            tuned = (int)tp.size();
            if (n == 1) {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                g_tune_cache[sig] = chosen;
            }
        }
        VPX_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        // an error part-way leaves every pass on its default choice
        for (TunePass &t : tp) gemm_set_choice(*t.call.g, t.dflt);
        for (int i = 0; i < n; ++i) ++plans[i]->tune_epoch;
        release();
        throw;
    }
    release();
    for (int i = 0; i < n; ++i) ++plans[i]->tune_epoch;   // later executes capture with the choices
    if (n_passes) *n_passes = tuned;
    if (n_changed) *n_changed = changed;
}

int device_sync_status(vpx_plan *p) {
    cudaStream_t s = (cudaStream_t)p->last_stream;
    VPX_CUDA(cudaStreamSynchronize(s));
    if (p->timing && p->events[0]) {
        VPX_CUDA(cudaStreamSynchronize((cudaStream_t)p->aux_stream));
        VPX_CUDA(cudaStreamSynchronize((cudaStream_t)p->aux2_stream));
        for (int i = 0; i < VPX_N_PASSES; ++i) {
            float ms = 0.f;
            if (p->events[i] && p->events[i + 1] &&
                cudaEventElapsedTime(&ms, (cudaEvent_t)p->events[i], (cudaEvent_t)p->events[i + 1]) == cudaSuccess) {
                p->pass_ms[i] = ms;
            } else {
                p->pass_ms[i] = 0.0;
                (void)cudaGetLastError();   // an unrecorded pair is not an error of the plan
            }
        }
        // the near field runs on the auxiliary stream: its own pair of events
        float ms = 0.f;
        if (p->events[VPX_N_PASSES + 1] && p->events[VPX_N_PASSES + 2] &&
            cudaEventElapsedTime(&ms, (cudaEvent_t)p->events[VPX_N_PASSES + 1],
                                 (cudaEvent_t)p->events[VPX_N_PASSES + 2]) == cudaSuccess)
            p->pass_ms[6] = ms;
        else
            (void)cudaGetLastError();
    }
    int st = 0;
    VPX_CUDA(cudaMemcpy(&st, p->wk.status, sizeof(int), cudaMemcpyDeviceToHost));
    VPX_CUDA(cudaMemset(p->wk.status, 0, sizeof(int)));
    return st;
}

void device_execute_host(vpx_plan *p, const double *f, int nrhs, double *v, double *vb) {
    const int64_t ns = (int64_t)p->stencil_xy.size() / 2, nt = (int64_t)p->leaf_xy.size() / 2;
    const int64_t nbd = (int64_t)p->bdry_xy.size() / 2;
    DevWork &w = p->wk;
    if (!w.f_tmp) {
        w.f_tmp = dev_alloc<double>((size_t)std::max<int64_t>(ns, 1) * w.max_rhs);
        w.v_tmp = dev_alloc<double>((size_t)nt * w.max_rhs);
        w.b_tmp = dev_alloc<double>((size_t)std::max<int64_t>(nbd, 1) * w.max_rhs);
    }
    cudaStream_t s = (cudaStream_t)p->stream;
    if (ns > 0) VPX_CUDA(cudaMemcpyAsync(w.f_tmp, f, sizeof(double) * ns * nrhs, cudaMemcpyHostToDevice, s));
    device_execute(p, w.f_tmp, nrhs, std::max<int64_t>(ns, 1), w.v_tmp, nt, nbd > 0 ? w.b_tmp : nullptr,
                   std::max<int64_t>(nbd, 1), s);
    VPX_CUDA(cudaMemcpyAsync(v, w.v_tmp, sizeof(double) * nt * nrhs, cudaMemcpyDeviceToHost, s));
    if (vb && nbd > 0) VPX_CUDA(cudaMemcpyAsync(vb, w.b_tmp, sizeof(double) * nbd * nrhs, cudaMemcpyDeviceToHost, s));
    VPX_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vpx
