// device_exec.cu -- the hot path: extension of f on cut leaves (Sections 3.2,
// 4.1) and the box FMM for the volume potential (eq. volinte) in FP64.
//
// Conventions (for every box B of side L at level l, centre c, half side h):
//   multipole  Phi(z) = a_0 log(z - c) + sum_{k>=1} at_k (L / (z - c))^k
//   local      Psi(z) = sum_{l>=0} bt_l ((z - c) / L)^l
//   V(x) = (1/2pi) Re Phi  (the complex log kernel; G = (1/2pi) log|x - y|).
// Leaf values are the K x K Gauss-Legendre node values of f^e on each leaf.
#include <cmath>

#include "dev_common.cuh"

namespace vpx {

constexpr double kInv2Pi = 0.15915494309189533576888376337251;

__device__ inline double box_side_d(int level) { return ldexp(1.0, -level); }

// ---------------------------------------------------------------- extension

// regular leaves: copy data; exterior leaves outside every extension list: 0
__global__ void k_leafvals(int n_leaves, int KK, const int32_t *leaf_cls, const int32_t *owner_flag,
                           const int64_t *reg_off, const double *f, int64_t ldf, double *fe, int64_t ldfe) {
    const int rhs = blockIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_leaves * KK) return;
    const int leaf = (int)(idx / KK), j = (int)(idx % KK);
    const int cls = leaf_cls[leaf];
    double *o = fe + rhs * ldfe + idx;
    if (cls == kRegular) *o = f[rhs * ldf + reg_off[leaf] + j];
    else if (cls == kExterior && owner_flag[leaf] == 0) *o = 0.0;
}

struct ExtArgs {
    int K, Kbar, NG;
    const int32_t *cut_leaf, *n_interior, *grid_src, *node_src, *owned_off, *owned;
    const int64_t *stencil_off, *pinv_off;
    const double *pinv, *A_grid, *cheb_inv, *tnodes;
    const int32_t *leaf_level, *leaf_ix, *leaf_iy;
    const double *f;
    int64_t ldf;
    double *fe;
    int64_t ldfe;
};

// One block per (cut leaf, rhs).  c = A_I^+ f_I; the Kbar x Kbar Chebyshev grid
// on Sbar takes the data at interior nodes and A_{Xbar^E,G} c at exterior
// nodes; its Chebyshev coefficients truncated to m + n < Kbar (eq.
// chebexpbarS) are evaluated at the cut leaf's exterior nodes and at all nodes
// of the exterior leaves in its extension list.
__global__ void k_extend(ExtArgs a) {
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
    // c = P_S f_I : one warp per row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const double *P = a.pinv + a.pinv_off[c];
    for (int k = warp; k < NG; k += nwarp) {
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

// ------------------------------------------------------------------- L2M

// mpole[box] = h^2 Q f  (rows 2k, 2k+1 = Re, Im of at_k; row 0 = a_0)
__global__ void k_l2m(int KK, int P, const int32_t *nz_leaves, const int32_t *leaf_box, const int32_t *leaf_level,
                      const double *l2m, const double *fe, int64_t ldfe, double *mpole, int64_t ldm) {
    extern __shared__ double sf[];
    const int leaf = nz_leaves[blockIdx.x], rhs = blockIdx.y;
    const double *f = fe + rhs * ldfe + (int64_t)leaf * KK;
    for (int j = threadIdx.x; j < KK; j += blockDim.x) sf[j] = f[j];
    __syncthreads();
    const double h = 0.5 * box_side_d(leaf_level[leaf]);
    double *m = mpole + rhs * ldm + (int64_t)leaf_box[leaf] * 2 * P;
    for (int row = threadIdx.x; row < 2 * P; row += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < KK; ++j) s += l2m[(size_t)j * 2 * P + row] * sf[j];
        m[row] = h * h * s;
    }
}

// ------------------------------------------------------------------- M2M

__global__ void k_m2m(int first, int count, int P, const int32_t *child0, const uint8_t *box_nz, const double *m2m,
                      double *mpole, int64_t ldm) {
    const int b = first + blockIdx.x, rhs = blockIdx.y;
    if (blockIdx.x >= count) return;
    const int c0 = child0[b];
    double *mp = mpole + rhs * ldm;
    if (c0 < 0 || !box_nz[b]) return;
    for (int l = threadIdx.x; l < P; l += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int c = 0; c < 4; ++c) {
            const int ch = c0 + c;
            if (!box_nz[ch]) continue;
            const double *a = mp + (int64_t)ch * 2 * P;
            const double *M = m2m + (size_t)c * P * P * 2;
            for (int k = 0; k <= l; ++k) {
                double mr = M[((size_t)k * P + l) * 2], mi = M[((size_t)k * P + l) * 2 + 1];
                double ar = a[2 * k], ai = a[2 * k + 1];
                sr += mr * ar - mi * ai;
                si += mr * ai + mi * ar;
            }
        }
        mp[(int64_t)b * 2 * P + 2 * l] = sr;
        mp[(int64_t)b * 2 * P + 2 * l + 1] = si;
    }
}

// ----------------------------------------------------------- M2L and S2L

struct M2LArgs {
    int P, KK, first, count;
    const int32_t *vlist, *xlist, *box_level, *leaf_level;
    const uint8_t *box_nz;
    const double *B;        // [P][P] real
    const double *pw;       // [40][P] complex: tau^-k, tau = offset / 2
    const double *s2l;      // [20][P][KK] complex
    const double *w2;       // [KK]
    const double *mpole, *fe;
    int64_t ldm, ldfe;
    double *local;
};

// One block per target box (levels >= 2); thread l accumulates bt_l.
// list i: u_k = at_k (-1/tau)^k ; v_l = sum_k B'_{lk} u_k ; bt_l += tau^-l v_l,
// plus the a_0 terms a_0 (log L + log|t|) and -a_0 / (l t^l), t = 2 tau.
// list i+: bt_l += H^2 sum_j S2L_c[l][j] f_j (+ H^2 log H sum_j w_j f_j for l = 0).
__global__ void k_m2l(M2LArgs a) {
    extern __shared__ double sm[];
    const int P = a.P;
    double *sB = sm;                 // P*P
    double *su = sB + P * P;         // 2P
    double *sf = su + 2 * P;         // KK
    const int rhs = blockIdx.y;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) sB[i] = a.B[i];
    const double *mp = a.mpole + rhs * a.ldm;
    for (int bi = blockIdx.x; bi < a.count; bi += gridDim.x) {
        const int b = a.first + bi;
        const int lev = a.box_level[b];
        const double L = box_side_d(lev);
        double accr = 0.0, acci = 0.0;
        const int l = threadIdx.x;
        for (int s = 0; s < kVSlots; ++s) {
            const int src = a.vlist[(size_t)b * kVSlots + s];
            if (src < 0) continue;      // uniform across the block
            __syncthreads();
            const double *am = mp + (int64_t)src * 2 * P;
            const double *pw = a.pw + (size_t)s * P * 2;
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                double ar = am[2 * k], ai = am[2 * k + 1];
                double pr = pw[2 * k], pi = pw[2 * k + 1];
                if (k & 1) {
                    pr = -pr;
                    pi = -pi;
                }
                su[2 * k] = (k == 0) ? 0.0 : ar * pr - ai * pi;
                su[2 * k + 1] = (k == 0) ? 0.0 : ar * pi + ai * pr;
            }
            __syncthreads();
            if (l < P) {
                double vr = 0.0, vi = 0.0;
                const double *Bl = sB + l * P;
                for (int k = 1; k < P; ++k) {
                    vr += Bl[k] * su[2 * k];
                    vi += Bl[k] * su[2 * k + 1];
                }
                const double pr = pw[2 * l], pi = pw[2 * l + 1];
                accr += pr * vr - pi * vi;
                acci += pr * vi + pi * vr;
                const double a0 = am[0];
                if (l == 0) {
                    // offset t from the slot index
                    int idx = 0, ox = 0, oy = 0;
                    for (int y = -3; y <= 3; ++y)
                        for (int x = -3; x <= 3; ++x) {
                            if (x >= -1 && x <= 1 && y >= -1 && y <= 1) continue;
                            if (idx == s) {
                                ox = x;
                                oy = y;
                            }
                            ++idx;
                        }
                    accr += a0 * (log(L) + 0.5 * log((double)(ox * ox + oy * oy)));
                } else {
                    const double sc = -a0 * ldexp(1.0, -l) / l;   // -a_0 / (l t^l) = -a_0 2^-l tau^-l / l
                    accr += sc * pr;
                    acci += sc * pi;
                }
            }
        }
        for (int s = 0; s < kXSlots; ++s) {
            const int src = a.xlist[(size_t)b * kXSlots + s];
            if (src < 0) continue;
            __syncthreads();
            const double *f = a.fe + rhs * a.ldfe + (int64_t)src * a.KK;
            for (int j = threadIdx.x; j < a.KK; j += blockDim.x) sf[j] = f[j];
            __syncthreads();
            if (l < P) {
                const double H = 0.5 * box_side_d(a.leaf_level[src]);
                const double *S = a.s2l + (size_t)s * a.KK * P * 2;
                double vr = 0.0, vi = 0.0;
                for (int j = 0; j < a.KK; ++j) {
                    vr += S[((size_t)j * P + l) * 2] * sf[j];
                    vi += S[((size_t)j * P + l) * 2 + 1] * sf[j];
                }
                if (l == 0) {
                    double w = 0.0;
                    for (int j = 0; j < a.KK; ++j) w += a.w2[j] * sf[j];
                    vr += log(H) * w;
                }
                accr += H * H * vr;
                acci += H * H * vi;
            }
        }
        if (l < P) {
            double *out = a.local + rhs * a.ldm + (int64_t)b * 2 * P;
            out[2 * l] = accr;
            out[2 * l + 1] = acci;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- L2L

__global__ void k_l2l(int first, int count, int P, const int32_t *box_parent, const int32_t *box_ix,
                      const int32_t *box_iy, const double *l2l, double *local, int64_t ldm) {
    if ((int)blockIdx.x >= count) return;
    const int b = first + blockIdx.x, rhs = blockIdx.y;
    const int par = box_parent[b];
    const int c = (box_ix[b] & 1) + 2 * (box_iy[b] & 1);
    double *lo = local + rhs * ldm;
    const double *pl = lo + (int64_t)par * 2 * P;
    for (int m = threadIdx.x; m < P; m += blockDim.x) {
        double sr = lo[(int64_t)b * 2 * P + 2 * m], si = lo[(int64_t)b * 2 * P + 2 * m + 1];
        const double *M = l2l + (size_t)c * P * P * 2;
        for (int l = m; l < P; ++l) {
            double mr = M[((size_t)l * P + m) * 2], mi = M[((size_t)l * P + m) * 2 + 1];
            double ar = pl[2 * l], ai = pl[2 * l + 1];
            sr += mr * ar - mi * ai;
            si += mr * ai + mi * ar;
        }
        lo[(int64_t)b * 2 * P + 2 * m] = sr;
        lo[(int64_t)b * 2 * P + 2 * m + 1] = si;
    }
}

// -------------------------------------------------- L2T, M2T, near log term

struct FarArgs {
    int K, KK, P;
    const int32_t *leaf_box, *leaf_level, *leaf_ix, *leaf_iy, *near, *wlist, *box_level, *box_ix, *box_iy;
    const double *l2t, *tnodes, *mpole, *local;
    int64_t ldm;
    double *v;
    int64_t ldv;
    int *status;
};

// One block per (leaf, rhs), thread i = target node.  Writes
// V_i = (1/2pi) [Re Psi(z_i) + sum_near log(h_s) a_0(s) + sum_{W in list i-} Re Phi_W(z_i)].
__global__ void k_leaf_far(FarArgs a) {
    extern __shared__ double sm[];
    const int P = a.P, KK = a.KK, K = a.K;
    double *sl = sm;            // 2P local
    double *sw = sl + 2 * P;    // 2P multipole of a list i- box
    double *snl = sw + 2 * P;   // 1
    const int leaf = blockIdx.x, rhs = blockIdx.y;
    const int box = a.leaf_box[leaf];
    const double *lo = a.local + rhs * a.ldm + (int64_t)box * 2 * P;
    const double *mp = a.mpole + rhs * a.ldm;
    const int lev = a.box_level[box];
    for (int q = threadIdx.x; q < 2 * P; q += blockDim.x) sl[q] = (lev >= 2) ? lo[q] : 0.0;
    __shared__ double s_nl[kNearConfigs];
    if (threadIdx.x < kNearConfigs) {
        int src = a.near[(size_t)leaf * kNearConfigs + threadIdx.x];
        double v = 0.0;
        if (src >= 0) v = log(0.5 * box_side_d(a.leaf_level[src])) * mp[(int64_t)a.leaf_box[src] * 2 * P];
        s_nl[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int c = 0; c < kNearConfigs; ++c) s += s_nl[c];
        snl[0] = s;
    }
    __syncthreads();
    const double sT = box_side_d(lev);
    const double cx = -0.5 + (a.leaf_ix[leaf] + 0.5) * sT, cy = -0.5 + (a.leaf_iy[leaf] + 0.5) * sT;
    double val = 0.0, zx = 0.0, zy = 0.0;
    const int i = threadIdx.x;
    if (i < KK) {
        for (int q = 0; q < 2 * P; ++q) val += a.l2t[(size_t)q * KK + i] * sl[q];
        val += snl[0];
        zx = cx + 0.5 * sT * a.tnodes[i % K];
        zy = cy + 0.5 * sT * a.tnodes[i / K];
    }
    for (int s = 0; s < kWSlots; ++s) {
        const int wb = a.wlist[(size_t)leaf * kWSlots + s];
        if (wb < 0) continue;
        __syncthreads();
        for (int q = threadIdx.x; q < 2 * P; q += blockDim.x) sw[q] = mp[(int64_t)wb * 2 * P + q];
        __syncthreads();
        if (i < KK) {
            const double LW = box_side_d(a.box_level[wb]);
            const double wx = -0.5 + (a.box_ix[wb] + 0.5) * LW, wy = -0.5 + (a.box_iy[wb] + 0.5) * LW;
            const double dx = zx - wx, dy = zy - wy, r2 = dx * dx + dy * dy;
            const double ur = LW * dx / r2, ui = -LW * dy / r2;   // L_W / (z - c_W)
            double hr = 0.0, hi = 0.0;                           // Horner: sum_{k>=1} at_k u^k
            for (int k = P - 1; k >= 1; --k) {
                double tr = hr + sw[2 * k], ti = hi + sw[2 * k + 1];
                hr = tr * ur - ti * ui;
                hi = tr * ui + ti * ur;
            }
            val += hr + sw[0] * 0.5 * log(r2);
        }
    }
    if (i < KK) {
        val *= kInv2Pi;
        if (!isfinite(val)) set_status(a.status, VPX_ERR_NAN);
        a.v[rhs * a.ldv + (int64_t)leaf * KK + i] = val;
    }
}

// ------------------------------------------------------ near-field GEMM

// Grouped GEMM: for every pair (target t, source s) of configuration c,
// V_t += (h_s^2 / 2pi) T_c f_s.  A CTA computes a 64 x 64 tile (64 target
// rows of T_c times the source vectors of 64 pairs), accumulating in
// registers (4 x 4 per thread), then adds into V with FP64 atomics.
constexpr int NB_M = 64, NB_N = 64, NB_K = 16;

__global__ void __launch_bounds__(256) k_near_fp64(int KK, const NearTile *tiles, const int32_t *tgt,
                                                   const int32_t *src, const int32_t *leaf_level, const double *tab,
                                                   const double *fe, int64_t ldfe, double *v, int64_t ldv) {
    __shared__ double As[NB_K][NB_M + 1];
    __shared__ double Bs[NB_K][NB_N + 1];
    const NearTile tile = tiles[blockIdx.x];
    const int m0 = blockIdx.y * NB_M, rhs = blockIdx.z;
    const double *A = tab + (size_t)tile.config * KK * KK;
    const double *F = fe + rhs * ldfe;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < KK; k0 += NB_K) {
        for (int e = threadIdx.x; e < NB_M * NB_K; e += 256) {
            int r = e / NB_K, k = e % NB_K;
            As[k][r] = (m0 + r < KK && k0 + k < KK) ? A[(size_t)(m0 + r) * KK + k0 + k] : 0.0;
        }
        for (int e = threadIdx.x; e < NB_N * NB_K; e += 256) {
            int n = e / NB_K, k = e % NB_K;
            Bs[k][n] = (n < tile.count && k0 + k < KK) ? F[(int64_t)src[tile.first + n] * KK + k0 + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NB_K; ++k) {
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
        int p = tile.first + n;
        double h = 0.5 * box_side_d(leaf_level[src[p]]);
        double sc = h * h * kInv2Pi;
        double *o = v + rhs * ldv + (int64_t)tgt[p] * KK;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = m0 + ty * 4 + i;
            if (r < KK) atomicAdd(o + r, sc * acc[i][j]);
        }
    }
}

// ---------------------------------------------------------------- boundary

__global__ void k_boundary(int nb, int K, const int32_t *bleaf, const double *bw, const double *v, int64_t ldv,
                           double *vb, int64_t ldb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, rhs = blockIdx.y;
    if (k >= nb) return;
    const double *w = bw + (size_t)k * 2 * K;
    const double *V = v + rhs * ldv + (int64_t)bleaf[k] * K * K;
    double s = 0.0;
    for (int b = 0; b < K; ++b) {
        double r = 0.0;
        for (int a2 = 0; a2 < K; ++a2) r += w[a2] * V[b * K + a2];
        s += w[K + b] * r;
    }
    vb[rhs * ldb + k] = s;
}

// ------------------------------------------------------------ host side

void setup_near_pairs(vpx_plan *p) {
    const int nl = (int)p->tree.leaves.size();
    std::vector<std::vector<std::pair<int32_t, int32_t>>> by(kNearConfigs);
    for (int t = 0; t < nl; ++t)
        for (int c = 0; c < kNearConfigs; ++c) {
            int s = p->near[(size_t)t * kNearConfigs + c];
            if (s >= 0) by[c].push_back({t, s});
        }
    std::vector<int32_t> tg, sr;
    std::vector<NearTile> tiles;
    for (int c = 0; c < kNearConfigs; ++c) {
        int first = (int)tg.size();
        for (auto &pr : by[c]) {
            tg.push_back(pr.first);
            sr.push_back(pr.second);
        }
        for (int i = 0; i < (int)by[c].size(); i += NB_N)
            tiles.push_back({c, first + i, std::min(NB_N, (int)by[c].size() - i)});
    }
    p->wk.near_tgt = dev_upload(tg);
    p->wk.near_src = dev_upload(sr);
    p->wk.near_tiles = dev_upload(tiles);
    p->wk.n_near_tiles = (int)tiles.size();
    p->wk.n_near_pairs = (int64_t)tg.size();
    std::vector<int32_t> nz;
    for (int i = 0; i < nl; ++i)
        if (p->leaf_nz[i]) nz.push_back(i);
    p->wk.nz_leaves = dev_upload(nz);
    p->wk.n_nz_leaves = (int)nz.size();
    // owner flag per leaf (exterior leaves inside an extension list)
    std::vector<int32_t> of(nl, 0);
    for (int i = 0; i < nl; ++i) of[i] = p->tree.leaves[i].owner >= 0 ? 1 : 0;
    p->ext.owned_flag_dev = dev_upload(of);
    // M2L: tau^-k for the 40 list-i offsets, tau = (dx + i dy) / 2
    const int P = p->P;
    std::vector<double> pw((size_t)kVSlots * P * 2);
    int idx = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            if (x >= -1 && x <= 1 && y >= -1 && y <= 1) continue;
            // tau = (x + i y) / 2 ; store tau^-k
            double tr = 0.5 * x, ti = 0.5 * y, n2 = tr * tr + ti * ti;
            double ir = tr / n2, ii = -ti / n2;   // 1/tau
            double cr = 1.0, ci = 0.0;
            for (int k = 0; k < P; ++k) {
                pw[((size_t)idx * P + k) * 2] = cr;
                pw[((size_t)idx * P + k) * 2 + 1] = ci;
                double nr = cr * ir - ci * ii;
                ci = cr * ii + ci * ir;
                cr = nr;
            }
            ++idx;
        }
    p->ext.m2l_pw = dev_upload(pw);
}

static void ev_record(vpx_plan *p, int i, cudaStream_t s) {
    if (!p->timing) return;
    if (!p->events[i]) VPX_CUDA(cudaEventCreate((cudaEvent_t *)&p->events[i]));
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->events[i], s));
}

static void run_extension(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *fe, int64_t ldfe,
                          cudaStream_t s) {
    const int nl = p->dt.n_leaves, KK = p->KK;
    const int64_t n = (int64_t)nl * KK;
    if (n > 0) {
        dim3 g((unsigned)((n + 255) / 256), nrhs);
        k_leafvals<<<g, 256, 0, s>>>(nl, KK, p->dt.leaf_cls, p->ext.owned_flag_dev, p->ext.reg_leaf_off, f, ldf, fe,
                                     ldfe);
        VPX_LAUNCH("k_leafvals");
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
        int maxI = 0;
        for (int c = 0; c < p->ext.ncut; ++c) maxI = std::max(maxI, st.n_interior[c]);
        size_t smem = sizeof(double) * ((size_t)maxI + st.NG + 3 * st.Kbar * st.Kbar + 3 * p->K * st.Kbar);
        if (smem > 48 * 1024) VPX_CUDA(cudaFuncSetAttribute(k_extend, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_extend<<<dim3(p->ext.ncut, nrhs), 256, smem, s>>>(a);
        VPX_LAUNCH("k_extend");
    }
}

// The passes of the box FMM with the multipole and local expansions in the
// scratch arrays mp and lo (each nrhs x n_boxes x 2P doubles).
void run_potential_scratch(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                           int64_t ldb, double *mp, double *lo, cudaStream_t s) {
    const int P = p->P, KK = p->KK, K = p->K;
    const DevTree &d = p->dt;
    const int64_t ldm = (int64_t)d.n_boxes * 2 * P;
    ev_record(p, 1, s);
    if (p->wk.n_nz_leaves > 0) {
        k_l2m<<<dim3(p->wk.n_nz_leaves, nrhs), 128, KK * sizeof(double), s>>>(
            KK, P, p->wk.nz_leaves, d.leaf_box, p->ext.leaf_level, p->tab.l2m, fe, ldfe, mp, ldm);
        VPX_LAUNCH("k_l2m");
    }
    ev_record(p, 2, s);
    for (int l = d.n_levels - 2; l >= 2; --l) {
        int first = d.level_start[l], count = d.level_start[l + 1] - first;
        if (count <= 0) continue;
        k_m2m<<<dim3(count, nrhs), 64, 0, s>>>(first, count, P, d.box_child0, d.box_nz, p->tab.m2m, mp, ldm);
        VPX_LAUNCH("k_m2m");
    }
    ev_record(p, 3, s);
    int first2 = d.level_start[std::min(2, d.n_levels)], count2 = d.n_boxes - first2;
    if (count2 > 0) {
        M2LArgs a;
        a.P = P;
        a.KK = KK;
        a.first = first2;
        a.count = count2;
        a.vlist = d.vlist;
        a.xlist = d.xlist;
        a.box_level = d.box_level;
        a.leaf_level = p->ext.leaf_level;
        a.box_nz = d.box_nz;
        a.B = p->tab.m2l_b;
        a.pw = p->ext.m2l_pw;
        a.s2l = p->tab.s2l;
        a.w2 = p->tab.w2;
        a.mpole = mp;
        a.fe = fe;
        a.ldm = ldm;
        a.ldfe = ldfe;
        a.local = lo;
        size_t smem = sizeof(double) * ((size_t)P * P + 2 * P + KK);
        if (smem > 48 * 1024) VPX_CUDA(cudaFuncSetAttribute(k_m2l, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int grid = std::min(count2, 152 * 8);
        k_m2l<<<dim3(grid, nrhs), 64, smem, s>>>(a);
        VPX_LAUNCH("k_m2l");
    }
    ev_record(p, 4, s);
    for (int l = 2; l + 1 < d.n_levels; ++l) {
        int first = d.level_start[l + 1], count = d.level_start[l + 2] - first;
        if (count <= 0) continue;
        k_l2l<<<dim3(count, nrhs), 64, 0, s>>>(first, count, P, d.box_parent, d.box_ix, d.box_iy, p->tab.l2l, lo, ldm);
        VPX_LAUNCH("k_l2l");
    }
    ev_record(p, 5, s);
    {
        FarArgs a;
        a.K = K;
        a.KK = KK;
        a.P = P;
        a.leaf_box = d.leaf_box;
        a.leaf_level = p->ext.leaf_level;
        a.leaf_ix = p->ext.leaf_ix;
        a.leaf_iy = p->ext.leaf_iy;
        a.near = d.near;
        a.wlist = d.wlist;
        a.box_level = d.box_level;
        a.box_ix = d.box_ix;
        a.box_iy = d.box_iy;
        a.l2t = p->tab.l2t;
        a.tnodes = p->tab.tnodes;
        a.mpole = mp;
        a.local = lo;
        a.ldm = ldm;
        a.v = v;
        a.ldv = ldv;
        a.status = p->wk.status;
        size_t smem = sizeof(double) * (4 * P + 1);
        k_leaf_far<<<dim3(d.n_leaves, nrhs), std::max(64, ((KK + 31) / 32) * 32), smem, s>>>(a);
        VPX_LAUNCH("k_leaf_far");
    }
    ev_record(p, 6, s);
    if (p->wk.n_near_tiles > 0) {
        dim3 g(p->wk.n_near_tiles, (KK + NB_M - 1) / NB_M, nrhs);
        k_near_fp64<<<g, 256, 0, s>>>(KK, p->wk.near_tiles, p->wk.near_tgt, p->wk.near_src, p->ext.leaf_level,
                                     p->tab.near, fe, ldfe, v, ldv);
        VPX_LAUNCH("k_near_fp64");
    }
    ev_record(p, 7, s);
    const int nbd = (int)p->bdry_leaf.size();
    if (vb && nbd > 0) {
        k_boundary<<<dim3((nbd + 127) / 128, nrhs), 128, 0, s>>>(nbd, K, p->wk.bdry_leaf, p->wk.bdry_w, v, ldv, vb,
                                                                ldb);
        VPX_LAUNCH("k_boundary");
    }
    ev_record(p, 8, s);
}

static void run_potential(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                          int64_t ldb, cudaStream_t s) {
    run_potential_scratch(p, fe, ldfe, nrhs, v, ldv, vb, ldb, p->wk.mpole, p->wk.local, s);
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

void device_execute(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *v, int64_t ldv, double *vb,
                    int64_t ldb, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = stream;
    const int64_t ldfe = (int64_t)p->dt.n_leaves * p->KK;
    ev_record(p, 0, s);
    run_extension(p, f, nrhs, ldf, p->wk.fe, ldfe, s);
    run_potential(p, p->wk.fe, ldfe, nrhs, v, ldv, vb, ldb, s);
}

int device_sync_status(vpx_plan *p) {
    cudaStream_t s = (cudaStream_t)p->last_stream;
    VPX_CUDA(cudaStreamSynchronize(s));
    if (p->timing && p->events[0]) {
        for (int i = 0; i < VPX_N_PASSES; ++i) {
            float ms = 0.f;
            if (p->events[i] && p->events[i + 1] &&
                cudaEventElapsedTime(&ms, (cudaEvent_t)p->events[i], (cudaEvent_t)p->events[i + 1]) == cudaSuccess)
                p->pass_ms[i] = ms;
            else
                p->pass_ms[i] = 0.0;
        }
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
