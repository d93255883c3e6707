// bie_device.cu -- device part of the boundary correction (Section 5, and
// Section 2 for domains with holes and exterior problems).
//
// Unknowns: the density sigma at the N boundary nodes, then one coefficient
// A_k per log term log|x - s_k| (one per hole, or one per inclusion of an
// exterior problem).  Rows: the boundary condition at every node,
//
//   jump_a sigma_a + sum_b D_ab sigma_b [+ (1/2pi) sum_b s_b w_b sigma_b]
//                  + sum_k A_k log|y_a - s_k| = g_a - V_a,
//
// (the bracket for exterior problems), then one constraint per log term:
// zero circulation int sigma ds = 0 on each hole; for an exterior problem on
// every inclusion but the last, and sum_k A_k = growth in the last row.  D is
// the double layer of eq. dblker on the panels' Gauss-Legendre nodes, with
// -kappa/(4pi) s w on its diagonal (eq. discdblpotpanel).
//
// The system depends on the geometry only, so it is assembled and inverted
// once (Gauss-Jordan with partial pivoting, one pivot column per step); a
// solve is then one matrix-vector product, read row by row by warps.  The
// evaluation sums the kernel over all boundary nodes for every leaf node in
// FP64 (sources staged through shared memory in tiles), adds the stored
// product-integration corrections of the panels near that node, the log
// terms and, for exterior problems, the constant (1/2pi) int sigma ds.
#include <cmath>

#include "dev_common.cuh"

namespace vpx {

namespace {

constexpr int kTile = 256;

__global__ void k_bie_assemble(int N, int n_log, int ntot, int exterior, const double *y, const double *nu,
                               const double *sw, const double *kappa, const double *jump, const int32_t *curve,
                               const double *log_c, const int32_t *log_curve, double *aug) {
    const int64_t ld = 2 * (int64_t)ntot;
    const int64_t total = (int64_t)ntot * ntot;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ntot), j = (int)(e % ntot);
        double v = 0.0;
        if (i < N) {
            if (j < N) {
                if (i == j) {
                    v = jump[i] - kappa[i] / (4.0 * M_PI) * sw[i];
                } else {
                    const double dx = y[2 * i] - y[2 * j], dy = y[2 * i + 1] - y[2 * j + 1];
                    v = (dx * nu[2 * j] + dy * nu[2 * j + 1]) / (dx * dx + dy * dy) / (2.0 * M_PI) * sw[j];
                }
                if (exterior) v += sw[j] / (2.0 * M_PI);
            } else {
                const int k = j - N;
                v = log(hypot(y[2 * i] - log_c[2 * k], y[2 * i + 1] - log_c[2 * k + 1]));
            }
        } else {
            const int r = i - N;
            if (exterior && r == n_log - 1) {
                v = (j >= N) ? 1.0 : 0.0;
            } else if (j < N) {
                v = (curve[j] == log_curve[r]) ? sw[j] : 0.0;
            }
        }
        aug[i * ld + j] = v;
        aug[i * ld + ntot + j] = (i == j) ? 1.0 : 0.0;
    }
}

// pivot of column k: the row of largest magnitude among k..ntot-1 (the first
// of equal ones), its value; a zero column latches VPX_ERR_STATE, after which
// every kernel of the elimination returns at once (the setup then fails)
__global__ void __launch_bounds__(1024) k_gj_pivot(int ntot, int k, const double *aug, int *piv_row, double *piv_val,
                                                   int *status) {
    if (*(volatile int *)status != 0) return;
    const int64_t ld = 2 * (int64_t)ntot;
    __shared__ double sv[1024];
    __shared__ int si[1024];
    double best = -1.0;
    int bi = ntot;
    for (int i = k + (int)threadIdx.x; i < ntot; i += blockDim.x) {
        const double a = fabs(aug[i * ld + k]);
        if (a > best) {
            best = a;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const double o = sv[threadIdx.x + s];
            const int oi = si[threadIdx.x + s];
            if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (!(sv[0] > 0.0) || si[0] >= ntot) {
            set_status(status, VPX_ERR_STATE);
            *piv_row = k;
            *piv_val = 1.0;
        } else {
            *piv_row = si[0];
            *piv_val = aug[si[0] * ld + k];
        }
    }
}

// rows k and p exchanged, the new row k divided by the pivot
__global__ void k_gj_swap(int ntot, int k, double *aug, const int *piv_row, const double *piv_val, const int *status) {
    if (*(const volatile int *)status != 0) return;
    const int64_t ld = 2 * (int64_t)ntot;
    const int p = *piv_row;
    const double pv = *piv_val;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ld; j += (int64_t)gridDim.x * blockDim.x) {
        const double a = aug[k * ld + j], b = aug[(int64_t)p * ld + j];
        aug[k * ld + j] = b / pv;
        if (p != k) aug[(int64_t)p * ld + j] = a;
    }
}

__global__ void k_gj_factors(int ntot, int k, const double *aug, double *fac, const int *status) {
    if (*(const volatile int *)status != 0) return;
    const int64_t ld = 2 * (int64_t)ntot;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += gridDim.x * blockDim.x)
        fac[i] = (i == k) ? 0.0 : aug[(int64_t)i * ld + k];
}

// every other row minus its multiple of row k; columns left of k are already
// unit vectors, and row k vanishes there
__global__ void k_gj_eliminate(int ntot, int k, double *aug, const double *fac, const int *status) {
    if (*(const volatile int *)status != 0) return;
    const int64_t ld = 2 * (int64_t)ntot;
    const int64_t width = ld - k;
    const int64_t total = (int64_t)ntot * width;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / width);
        const int64_t j = k + e % width;
        const double f = fac[i];
        if (f != 0.0) aug[(int64_t)i * ld + j] -= f * aug[(int64_t)k * ld + j];
    }
}

__global__ void k_bie_rhs(int N, int ntot, int exterior, const double *g, const double *vb, double growth, double *rhs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += gridDim.x * blockDim.x)
        rhs[i] = (i < N) ? g[i] - vb[i] : ((exterior && i == ntot - 1) ? growth : 0.0);
}

// y = M x, M row-major ntot x ntot: one warp per row
__global__ void __launch_bounds__(256) k_gemv_rows(int ntot, const double *M, const double *x, double *y) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= ntot) return;
    const double *m = M + (int64_t)row * ntot;
    double s = 0.0;
    for (int j = lane; j < ntot; j += 32) s += m[j] * x[j];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

// (1/2pi) sum_b s_b w_b sigma_b, one block
__global__ void __launch_bounds__(256) k_bie_const(int N, const double *sw, const double *sigma, double *out) {
    __shared__ double ws[8];
    double s = 0.0;
    for (int b = threadIdx.x; b < N; b += blockDim.x) s += sw[b] * sigma[b];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < 8 ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *out = s / (2.0 * M_PI);
    }
}

struct EvalArgs {
    int64_t nt;
    int N, nq, n_log;
    const double *tx;        // leaf nodes, 2 per node
    const double *y, *nu, *sw;
    const double *sol;       // sigma (N) then A_k (n_log)
    const int64_t *corr_off;
    const int32_t *corr_panel;
    const double *corr_w;
    const double *log_c;
    const double *cst;       // the exterior constant, or null
    const double *v;         // V at the leaf nodes
    double *u;
};

__global__ void __launch_bounds__(kTile) k_bie_eval(EvalArgs a) {
    __shared__ double s_y[2 * kTile], s_n[2 * kTile], s_q[kTile];
    const int64_t t = (int64_t)blockIdx.x * kTile + threadIdx.x;
    const bool live = t < a.nt;
    const double x = live ? a.tx[2 * t] : 0.0, yv = live ? a.tx[2 * t + 1] : 0.0;
    double acc = 0.0;
    for (int b0 = 0; b0 < a.N; b0 += kTile) {
        const int b = b0 + threadIdx.x;
        if (b < a.N) {
            s_y[2 * threadIdx.x] = a.y[2 * b];
            s_y[2 * threadIdx.x + 1] = a.y[2 * b + 1];
            s_n[2 * threadIdx.x] = a.nu[2 * b];
            s_n[2 * threadIdx.x + 1] = a.nu[2 * b + 1];
            s_q[threadIdx.x] = a.sw[b] * a.sol[b];
        }
        __syncthreads();
        const int nb = min(kTile, a.N - b0);
        for (int k = 0; k < nb; ++k) {
            const double dx = x - s_y[2 * k], dy = yv - s_y[2 * k + 1];
            const double r2 = dx * dx + dy * dy;
            if (r2 > 0.0) acc += (dx * s_n[2 * k] + dy * s_n[2 * k + 1]) / r2 * s_q[k];
        }
        __syncthreads();
    }
    if (!live) return;
    double u = acc / (2.0 * M_PI);
    for (int64_t e = a.corr_off[t]; e < a.corr_off[t + 1]; ++e) {
        const double *w = a.corr_w + e * a.nq;
        const double *sg = a.sol + (int64_t)a.corr_panel[e] * a.nq;
        for (int j = 0; j < a.nq; ++j) u += w[j] * sg[j];
    }
    for (int k = 0; k < a.n_log; ++k) u += a.sol[a.N + k] * log(hypot(x - a.log_c[2 * k], yv - a.log_c[2 * k + 1]));
    if (a.cst) u += *a.cst;
    a.u[t] = u + a.v[t];
}

}  // namespace

// Inverse of the n x n matrix held in the left half of aug (n x 2n, row-major,
// the right half the identity) by Gauss-Jordan with partial pivoting, one
// pivot column per step, into inv (n x n).  Returns 0, or VPX_ERR_STATE when a
// pivot column is zero (or not a number): the pivot kernel latches the status,
// every later kernel of the elimination returns at once, and the host loop
// stops at its next check (every 256 columns).  Synchronous.
int gauss_jordan_inverse(int ntot, double *aug, double *inv) {
    double *fac = dev_alloc<double>(ntot), *pv = dev_alloc<double>(1);
    int *pr = dev_alloc<int>(1), *status = dev_alloc<int>(1);
    VPX_CUDA(cudaMemset(status, 0, sizeof(int)));
    const int grid = 152 * 8;
    int st = 0;
    for (int k = 0; k < ntot; ++k) {
        k_gj_pivot<<<1, 1024>>>(ntot, k, aug, pr, pv, status);
        k_gj_swap<<<(2 * ntot + 255) / 256, 256>>>(ntot, k, aug, pr, pv, status);
        k_gj_factors<<<(ntot + 255) / 256, 256>>>(ntot, k, aug, fac, status);
        k_gj_eliminate<<<grid, 256>>>(ntot, k, aug, fac, status);
        if ((k & 255) == 255) {
            VPX_LAUNCH("Gauss-Jordan inversion");
            VPX_CUDA(cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost));
            if (st != 0) break;
        }
    }
    VPX_LAUNCH("Gauss-Jordan inversion");
    VPX_CUDA(cudaMemcpy2D(inv, sizeof(double) * ntot, aug + ntot, sizeof(double) * 2 * ntot, sizeof(double) * ntot,
                          ntot, cudaMemcpyDeviceToDevice));
    VPX_CUDA(cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost));
    dev_free(fac);
    dev_free(pv);
    dev_free(pr);
    dev_free(status);
    return st;
}

void device_bie_setup(vpx_plan *pl) {
    if (pl->device >= 0) VPX_CUDA(cudaSetDevice(pl->device));
    BieHost &B = pl->bie;
    const int N = (int)(pl->bdry_xy.size() / 2);
    const int ntot = N + B.n_log;
    B.n_unknowns = ntot;
    BieDev &d = B.dev;
    d.y = dev_upload(pl->bdry_xy);
    d.nu = dev_upload(B.nu);
    d.sw = dev_upload(B.sw);
    d.leaf_xy = dev_upload(pl->leaf_xy);
    d.corr_off = dev_upload(B.corr_off);
    d.corr_panel = dev_upload(B.corr_panel);
    d.corr_w = dev_upload(B.corr_w);
    d.log_c = dev_upload(B.log_centre);
    d.rhs = dev_alloc<double>(ntot);
    d.cst = dev_alloc<double>(1);
    d.minv = dev_alloc<double>((size_t)ntot * ntot);
    double *kappa = dev_upload(B.kappa), *jump = dev_upload(B.jump);
    int32_t *curve = dev_upload(B.curve_of_node), *log_curve = dev_upload(B.log_curve);
    double *aug = dev_alloc<double>((size_t)ntot * 2 * ntot);
    const int exterior = B.outer_curve < 0 ? 1 : 0;
    k_bie_assemble<<<152 * 8, 256>>>(N, B.n_log, ntot, exterior, d.y, d.nu, d.sw, kappa, jump, curve, d.log_c,
                                     log_curve, aug);
    VPX_LAUNCH("k_bie_assemble");
    const int st = gauss_jordan_inverse(ntot, aug, d.minv);
    dev_free(aug);
    dev_free(kappa);
    dev_free(jump);
    dev_free(curve);
    dev_free(log_curve);
    if (st != 0) fail(VPX_ERR_STATE, "the boundary-correction system is singular");
}

int device_check_gauss_jordan(int n, const double *a, double *inv) {
    double *aug = dev_alloc<double>((size_t)n * 2 * n), *out = dev_alloc<double>((size_t)n * n);
    std::vector<double> h((size_t)n * 2 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) h[(size_t)i * 2 * n + j] = a[(size_t)i * n + j];
        h[(size_t)i * 2 * n + n + i] = 1.0;
    }
    VPX_CUDA(cudaMemcpy(aug, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    const int st = gauss_jordan_inverse(n, aug, out);
    VPX_CUDA(cudaMemcpy(inv, out, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
    dev_free(aug);
    dev_free(out);
    return st;
}

void device_bie_solve(vpx_plan *pl, const double *g, const double *vb, double growth, double *sol, void *stream) {
    BieHost &B = pl->bie;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = (int)(pl->bdry_xy.size() / 2), ntot = B.n_unknowns;
    k_bie_rhs<<<(ntot + 255) / 256, 256, 0, s>>>(N, ntot, B.outer_curve < 0 ? 1 : 0, g, vb, growth, B.dev.rhs);
    VPX_LAUNCH("k_bie_rhs");
    k_gemv_rows<<<(ntot + 7) / 8, 256, 0, s>>>(ntot, B.dev.minv, B.dev.rhs, sol);
    VPX_LAUNCH("k_gemv_rows");
}

void device_bie_eval(vpx_plan *pl, const double *sol, const double *v, double *u, void *stream) {
    BieHost &B = pl->bie;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = (int)(pl->bdry_xy.size() / 2);
    const bool exterior = B.outer_curve < 0;
    if (exterior) {
        k_bie_const<<<1, 256, 0, s>>>(N, B.dev.sw, sol, B.dev.cst);
        VPX_LAUNCH("k_bie_const");
    }
    EvalArgs a;
    a.nt = (int64_t)(pl->leaf_xy.size() / 2);
    a.N = N;
    a.nq = B.nq;
    a.n_log = B.n_log;
    a.tx = B.dev.leaf_xy;
    a.y = B.dev.y;
    a.nu = B.dev.nu;
    a.sw = B.dev.sw;
    a.sol = sol;
    a.corr_off = B.dev.corr_off;
    a.corr_panel = B.dev.corr_panel;
    a.corr_w = B.dev.corr_w;
    a.log_c = B.dev.log_c;
    a.cst = exterior ? B.dev.cst : nullptr;
    a.v = v;
    a.u = u;
    k_bie_eval<<<(unsigned)((a.nt + kTile - 1) / kTile), kTile, 0, s>>>(a);
    VPX_LAUNCH("k_bie_eval");
}

void device_bie_free(vpx_plan *pl) {
    BieDev &d = pl->bie.dev;
    dev_free(d.y);
    dev_free(d.nu);
    dev_free(d.sw);
    dev_free(d.leaf_xy);
    dev_free(d.corr_off);
    dev_free(d.corr_panel);
    dev_free(d.corr_w);
    dev_free(d.log_c);
    dev_free(d.rhs);
    dev_free(d.cst);
    dev_free(d.minv);
}

}  // namespace vpx
