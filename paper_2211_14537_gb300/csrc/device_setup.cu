// device_setup.cu -- per-geometry setup on the GPU: the upload of the tree,
// its interaction lists (built on the device), near-field tables (polar
// quadrature), S2L tables and the small expansion/translation tables computed
// on the host.
#include <algorithm>
#include <cmath>
#include <complex>

#include "dev_common.cuh"

namespace vpx {

// ------------------------------------------------------ near-field tables
//
// T_c[i][j] = int_{[-1,1]^2} log|x_i - eta| l_j(eta) d eta, x_i the i-th target
// node in the reference coordinates of the source box, for the 33 relative
// configurations of a target leaf and a same-level, coarser or finer source
// leaf (Section 4: the near field is exact for the piecewise polynomial).
// Self configuration: polar coordinates about x_i on the four triangles
// (x_i, edge), exact radial rules, graded Gauss-Legendre panels along each
// edge.  Other configurations: admissible rectangles graded toward x_i.

struct NearGeom {
    double tau_x, tau_y, sigma;   // target box centre / half side in source units
};

constexpr int kNS = 20;           // Gauss-Legendre nodes per s-panel
constexpr int kMaxPanels = 96;

struct TableRules {
    double t[kMaxK], bary[kMaxK];              // leaf nodes, barycentric weights
    double rg[kMaxK], rgw[kMaxK];              // Gauss-Legendre on [0,1] (K nodes)
    double rl[kMaxK], rlw[kMaxK];              // Gauss rule for -rho log rho on [0,1]
    double sg[kNS], sgw[kNS];                  // Gauss-Legendre on [0,1] (s panels)
};

__device__ inline void d_lagrange(int K, const double *t, const double *bw, double s, double *out) {
    for (int a = 0; a < K; ++a)
        if (s == t[a]) {
            for (int m = 0; m < K; ++m) out[m] = (m == a) ? 1.0 : 0.0;
            return;
        }
    double den = 0.0;
    for (int a = 0; a < K; ++a) {
        out[a] = bw[a] / (s - t[a]);
        den += out[a];
    }
    double inv = 1.0 / den;
    for (int a = 0; a < K; ++a) out[a] *= inv;
}

// Self configuration only (the target node lies inside the source box, so
// every triangle (x_i, edge) lies inside the box).  One block per target node;
// K*K threads, thread j = basis function.
template <int K>
__global__ void __launch_bounds__(K * K) k_near_self(TableRules R, double *out) {
    constexpr int KK = K * K;
    constexpr int CH = 64 / K;              // s-nodes per chunk
    constexpr int NPT = CH * 2 * K;         // quadrature points per chunk (= 128)
    const int tgt = blockIdx.x;
    const int j = threadIdx.x;
    const int ja = j % K, jb = j / K;
    __shared__ double s_w[NPT], s_la[NPT][K], s_lb[NPT][K];
    __shared__ double s_pan[kMaxPanels + 1];
    __shared__ int s_npan;
    const double x = R.t[tgt % K];
    const double y = R.t[tgt / K];
    double acc = 0.0;
    const double P0x[4] = {-1, 1, 1, -1}, P0y[4] = {-1, -1, 1, 1};
    const double P1x[4] = {1, 1, -1, -1}, P1y[4] = {-1, 1, 1, -1};
    const double Nx[4] = {0, 1, 0, -1}, Ny[4] = {-1, 0, 1, 0};
    for (int e = 0; e < 4; ++e) {
        const double d = (P0x[e] - x) * Nx[e] + (P0y[e] - y) * Ny[e];   // > 0: x inside
        const double ex = P1x[e] - P0x[e], ey = P1y[e] - P0y[e];
        const double len = 2.0;
        if (threadIdx.x == 0) {
            double sf = ((x - P0x[e]) * ex + (y - P0y[e]) * ey) / (len * len);
            double sc = fmin(fmax(sf, 0.0), 1.0);
            double delta = fmax(fabs(d) / len, 1e-14);
            double bl[kMaxPanels], br[kMaxPanels];
            int nl = 0, nr = 0;
            for (double w = delta; sc - w > 0.0 && nl < kMaxPanels / 2 - 1; w *= 2.0) bl[nl++] = sc - w;
            for (double w = delta; sc + w < 1.0 && nr < kMaxPanels / 2 - 1; w *= 2.0) br[nr++] = sc + w;
            int n = 0;
            s_pan[n++] = 0.0;
            for (int i = nl - 1; i >= 0; --i) s_pan[n++] = bl[i];
            if (sc > 0.0 && sc < 1.0) s_pan[n++] = sc;
            for (int i = 0; i < nr; ++i) s_pan[n++] = br[i];
            s_pan[n++] = 1.0;
            s_npan = n - 1;
        }
        __syncthreads();
        const int nsn = s_npan * kNS;
        for (int c0 = 0; c0 < nsn; c0 += CH) {
            for (int pt = threadIdx.x; pt < NPT; pt += blockDim.x) {
                int q = c0 + pt / (2 * K), r = pt % (2 * K);
                double wgt = 0.0, px = 0.0, py = 0.0;
                if (q < nsn) {
                    int pan = q / kNS, k = q % kNS;
                    double a = s_pan[pan], b = s_pan[pan + 1];
                    double s = a + (b - a) * R.sg[k];
                    double ws = (b - a) * R.sgw[k];
                    double Px = P0x[e] + s * ex, Py = P0y[e] + s * ey;
                    double Rx = Px - x, Ry = Py - y;
                    double logR = 0.5 * log(Rx * Rx + Ry * Ry);
                    double rho, wr;
                    if (r < K) {
                        rho = R.rg[r];
                        wr = R.rgw[r] * rho * logR;           // int rho log R(s) (.)
                    } else {
                        rho = R.rl[r - K];
                        wr = -R.rlw[r - K];                   // int rho log rho (.)
                    }
                    wgt = d * len * ws * wr;
                    px = x + rho * Rx;
                    py = y + rho * Ry;
                }
                s_w[pt] = wgt;
                d_lagrange(K, R.t, R.bary, px, s_la[pt]);
                d_lagrange(K, R.t, R.bary, py, s_lb[pt]);
            }
            __syncthreads();
#pragma unroll 4
            for (int pt = 0; pt < NPT; ++pt) acc += s_w[pt] * s_la[pt][ja] * s_lb[pt][jb];
            __syncthreads();
        }
    }
    out[((size_t)4 * KK + tgt) * KK + j] = acc;   // configuration 4 = (dx, dy) = (0, 0)
}

// The 32 other configurations: the target node lies outside the source box.
// The box is covered by rectangles that are admissible for a 24-point tensor
// Gauss-Legendre rule (distance to the target >= their diagonal), generated on
// the host by dyadic subdivision toward the target; every quadrature point is
// inside the box, so the basis polynomials are never extrapolated.
struct Rect {
    double x0, x1, y0, y1;
};
constexpr int kRQ = 24;   // a degree K-1 basis times the kernel: 24 points for K <= 16

template <int K>
__global__ void __launch_bounds__(K * K) k_near_rects(const NearGeom *geom, const int32_t *roff, const Rect *rects,
                                                      TableRules R, const double *gq, const double *gqw, double *out) {
    constexpr int KK = K * K;
    constexpr int NPT = kRQ * kRQ;
    const int item = blockIdx.x;              // (cfg, tgt)
    const int cfg = item / KK, tgt = item % KK;
    if (cfg == 4) return;
    const int j = threadIdx.x, ja = j % K, jb = j / K;
    __shared__ double s_w[NPT];
    __shared__ double s_la[kRQ][K], s_lb[kRQ][K];
    const NearGeom g = geom[cfg];
    const double x = g.tau_x + g.sigma * R.t[tgt % K];
    const double y = g.tau_y + g.sigma * R.t[tgt / K];
    double acc = 0.0;
    for (int r = roff[item]; r < roff[item + 1]; ++r) {
        const Rect rc = rects[r];
        const double hx = 0.5 * (rc.x1 - rc.x0), hy = 0.5 * (rc.y1 - rc.y0);
        const double mx = 0.5 * (rc.x1 + rc.x0), my = 0.5 * (rc.y1 + rc.y0);
        for (int pt = threadIdx.x; pt < NPT; pt += blockDim.x) {
            int ix = pt % kRQ, iy = pt / kRQ;
            double px = mx + hx * gq[ix], py = my + hy * gq[iy];
            double dx = px - x, dy = py - y;
            s_w[pt] = hx * hy * gqw[ix] * gqw[iy] * 0.5 * log(dx * dx + dy * dy);
        }
        for (int i = threadIdx.x; i < 2 * kRQ; i += blockDim.x) {
            if (i < kRQ) d_lagrange(K, R.t, R.bary, mx + hx * gq[i], s_la[i]);
            else d_lagrange(K, R.t, R.bary, my + hy * gq[i - kRQ], s_lb[i - kRQ]);
        }
        __syncthreads();
        for (int iy = 0; iy < kRQ; ++iy) {
            double sacc = 0.0;
#pragma unroll
            for (int ix = 0; ix < kRQ; ++ix) sacc += s_w[iy * kRQ + ix] * s_la[ix][ja];
            acc += sacc * s_lb[iy][jb];
        }
        __syncthreads();
    }
    out[((size_t)cfg * KK + tgt) * KK + j] = acc;
}

static void rect_cover(double x, double y, double x0, double x1, double y0, double y1, int depth, std::vector<Rect> &out) {
    double dx = std::max(std::max(x0 - x, x - x1), 0.0), dy = std::max(std::max(y0 - y, y - y1), 0.0);
    double dist = std::sqrt(dx * dx + dy * dy), diam = std::hypot(x1 - x0, y1 - y0);
    if (dist >= diam || depth >= 40) {
        out.push_back({x0, x1, y0, y1});
        return;
    }
    double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
    rect_cover(x, y, x0, xm, y0, ym, depth + 1, out);
    rect_cover(x, y, xm, x1, y0, ym, depth + 1, out);
    rect_cover(x, y, x0, xm, ym, y1, depth + 1, out);
    rect_cover(x, y, xm, x1, ym, y1, depth + 1, out);
}

// ------------------------------------------------------------- S2L tables
//
// S2L_c[l][j] = int ell_j(eta) (-1)^{l+1} / (l (tau - eta)^l) d eta   (l >= 1)
// S2L_c[0][j] = int ell_j(eta) log|tau - eta| d eta
// for the 20 positions tau of a target box relative to a coarse source leaf
// (list i+); composite tensor Gauss-Legendre on [-1,1]^2 (smooth integrand).
constexpr int kS2LPanels = 4, kS2LNodes = 16;

template <int K>
__global__ void __launch_bounds__(K * K) k_s2l_tables(int P, TableRules R, const double *gl16, const double *gl16w,
                                                      double *out) {
    constexpr int KK = K * K;
    const int cfg = blockIdx.x / P, l = blockIdx.x % P;
    const int j = threadIdx.x, ja = j % K, jb = j / K;
    int idx = 0, rx = 0, ry = 0;
    for (int yy = -2; yy <= 3; ++yy)
        for (int xx = -2; xx <= 3; ++xx) {
            if (xx >= -1 && xx <= 2 && yy >= -1 && yy <= 2) continue;
            if (idx == cfg) {
                rx = xx;
                ry = yy;
            }
            ++idx;
        }
    const double tx = rx - 0.5, ty = ry - 0.5;
    constexpr int NP1 = kS2LPanels * kS2LNodes;
    __shared__ double s_la[NP1][K];
    __shared__ double s_x[NP1], s_w[NP1];
    for (int i = threadIdx.x; i < NP1; i += blockDim.x) {
        int pan = i / kS2LNodes, k = i % kS2LNodes;
        double a = -1.0 + 2.0 * pan / kS2LPanels, b = a + 2.0 / kS2LPanels;
        s_x[i] = 0.5 * (a + b) + 0.5 * (b - a) * gl16[k];
        s_w[i] = 0.5 * (b - a) * gl16w[k];
        d_lagrange(K, R.t, R.bary, s_x[i], s_la[i]);
    }
    __syncthreads();
    double ar = 0.0, ai = 0.0;
    for (int iy = 0; iy < NP1; ++iy) {
        double accr = 0.0, acci = 0.0;
        for (int ix = 0; ix < NP1; ++ix) {
            double ux = tx - s_x[ix], uy = ty - s_x[iy];   // tau - eta
            double w = s_w[ix] * s_la[ix][ja];
            if (l == 0) {
                accr += w * 0.5 * log(ux * ux + uy * uy);
            } else {
                // (-1)^{l+1} / (l * u^l), u = ux + i uy
                double r2 = ux * ux + uy * uy;
                double vr = ux / r2, vi = -uy / r2;      // 1/u
                double pr = 1.0, pi = 0.0;
                for (int k = 0; k < l; ++k) {
                    double nr = pr * vr - pi * vi;
                    pi = pr * vi + pi * vr;
                    pr = nr;
                }
                double sgn = (l % 2 == 1) ? 1.0 : -1.0;
                accr += w * sgn * pr / l;
                acci += w * sgn * pi / l;
            }
        }
        double wy = s_w[iy] * s_la[iy][jb];
        ar += wy * accr;
        ai += wy * acci;
    }
    size_t o = (((size_t)cfg * KK + j) * P + l) * 2;   // [config][j][l]: l fastest
    out[o] = ar;
    out[o + 1] = ai;
}

// ---------------------------------------------------- host-computed tables

static void near_geometry(std::vector<NearGeom> &g) {
    g.clear();
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) g.push_back({-2.0 * dx, -2.0 * dy, 1.0});   // colleague source at target + (dx, dy)
    for (int y = -1; y <= 2; ++y)                                                  // coarse source
        for (int x = -1; x <= 2; ++x) {
            if (x >= 0 && x <= 1 && y >= 0 && y <= 1) continue;
            g.push_back({x - 0.5, y - 0.5, 0.5});
        }
    for (int y = -1; y <= 2; ++y)                                                  // fine source
        for (int x = -1; x <= 2; ++x) {
            if (x >= 0 && x <= 1 && y >= 0 && y <= 1) continue;
            g.push_back({2.0 * (0.5 - x), 2.0 * (0.5 - y), 2.0});
        }
}

static void rules(int K, TableRules &R) {
    std::vector<double> t, tw, g, gw, rl, rlw;
    gauss_legendre(K, t, tw);
    std::vector<double> bw = barycentric_weights(t);
    gauss_legendre(K, g, gw);
    gauss_log_rule(K, rl, rlw);
    std::vector<double> s, sw;
    gauss_legendre(kNS, s, sw);
    for (int i = 0; i < K; ++i) {
        R.t[i] = t[i];
        R.bary[i] = bw[i];
        R.rg[i] = 0.5 * (g[i] + 1.0);
        R.rgw[i] = 0.5 * gw[i];
        R.rl[i] = rl[i];
        R.rlw[i] = rlw[i];
    }
    for (int i = 0; i < kNS; ++i) {
        R.sg[i] = 0.5 * (s[i] + 1.0);
        R.sgw[i] = 0.5 * sw[i];
    }
}

template <int K>
static void launch_tables(vpx_plan *p, const TableRules &R, const NearGeom *dgeom, const double *d16, const double *d16w,
                          const int32_t *droff, const Rect *drects, const double *dq, const double *dqw) {
    k_near_self<K><<<K * K, K * K>>>(R, p->tab.near);
    VPX_LAUNCH("k_near_self");
    k_near_rects<K><<<kNearConfigs * K * K, K * K>>>(dgeom, droff, drects, R, dq, dqw, p->tab.near);
    VPX_LAUNCH("k_near_rects");
    k_s2l_tables<K><<<kXSlots * p->P, K * K>>>(p->P, R, d16, d16w, p->tab.s2l);
    VPX_LAUNCH("k_s2l_tables");
}

void setup_tables(vpx_plan *p) {
    const int K = p->K, KK = p->KK, P = p->P;
    TableRules R;
    rules(K, R);
    std::vector<NearGeom> geom;
    near_geometry(geom);
    NearGeom *dgeom = dev_upload(geom);
    std::vector<double> g16, g16w;
    gauss_legendre(kS2LNodes, g16, g16w);
    double *d16 = dev_upload(g16), *d16w = dev_upload(g16w);
    std::vector<double> gq, gqw;
    gauss_legendre(kRQ, gq, gqw);
    double *dq = dev_upload(gq), *dqw = dev_upload(gqw);
    std::vector<int32_t> roff{0};
    std::vector<Rect> rects;
    for (int c = 0; c < kNearConfigs; ++c)
        for (int i = 0; i < KK; ++i) {
            if (c != 4) {
                double x = geom[c].tau_x + geom[c].sigma * R.t[i % K];
                double y = geom[c].tau_y + geom[c].sigma * R.t[i / K];
                rect_cover(x, y, -1.0, 1.0, -1.0, 1.0, 0, rects);
            }
            roff.push_back((int32_t)rects.size());
        }
    int32_t *droff = dev_upload(roff);
    Rect *drects = dev_upload(rects);
    p->tab.near = dev_alloc<double>((size_t)kNearConfigs * KK * KK);
    p->tab.s2l = dev_alloc<double>((size_t)kXSlots * P * KK * 2);
    switch (K) {
        case 4: launch_tables<4>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        case 6: launch_tables<6>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        case 8: launch_tables<8>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        case 10: launch_tables<10>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        case 12: launch_tables<12>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        case 14: launch_tables<14>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        case 16: launch_tables<16>(p, R, dgeom, d16, d16w, droff, drects, dq, dqw); break;
        default: fail(VPX_ERR_ARG, "unsupported K");
    }
    VPX_CUDA(cudaDeviceSynchronize());
    dev_free(dgeom);
    dev_free(d16);
    dev_free(d16w);
    dev_free(dq);
    dev_free(dqw);
    dev_free(droff);
    dev_free(drects);
    std::vector<double> tq, tw, w2(KK);
    gauss_legendre(K, tq, tw);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a) w2[b * K + a] = tw[a] * tw[b];
    p->tab.w2 = dev_upload(w2);
    std::vector<double> t(R.t, R.t + K), bw(R.bary, R.bary + K);
    p->tab.tnodes = dev_upload(t);
    p->tab.bary = dev_upload(bw);
}

// --------------------------------------------------------------- uploads

void setup_near_pairs(vpx_plan *p);   // device_exec.cu
void build_lists_device(vpx_plan *p, cudaStream_t s);   // lists_device.cu
void setup_passes(vpx_plan *p);       // fmm_passes.cu
void free_passes(vpx_plan *p);

void device_setup(vpx_plan *p) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) fail(VPX_ERR_NODEV, "no CUDA device");
    VPX_CUDA(cudaGetDevice(&p->device));
    cudaStream_t s, aux, aux2;
    VPX_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    p->stream = s;
    VPX_CUDA(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking));
    p->aux_stream = aux;
    VPX_CUDA(cudaStreamCreateWithFlags(&aux2, cudaStreamNonBlocking));
    p->aux2_stream = aux2;
    for (void **e : {&p->ev_fork, &p->ev_up, &p->ev_join, &p->ev_join2, &p->ev_lc, &p->ev_lvf, &p->ev_lv,
                     &p->ev_bfork, &p->ev_bjoin})
        VPX_CUDA(cudaEventCreateWithFlags((cudaEvent_t *)e, cudaEventDisableTiming));
    DevTree &d = p->dt;
    d.n_leaves = (int)p->tree.leaves.size();
    d.n_boxes = (int)p->box_level.size();
    d.n_levels = p->n_levels;
    std::copy(p->level_start, p->level_start + kMaxLevel + 2, d.level_start);
    d.box_level = dev_upload(p->box_level);
    d.box_ix = dev_upload(p->box_ix);
    d.box_iy = dev_upload(p->box_iy);
    d.box_parent = dev_upload(p->box_parent);
    d.box_child0 = dev_upload(p->box_child0);
    d.box_leaf = dev_upload(p->box_leaf);
    d.box_morton = dev_upload(p->box_morton);
    d.box_nz = dev_upload(p->box_nz);
    d.leaf_nz = dev_upload(p->leaf_nz);
    std::vector<int32_t> leaf_box(d.n_leaves), lcls(d.n_leaves), llev(d.n_leaves), lix(d.n_leaves), liy(d.n_leaves);
    for (int b = 0; b < d.n_boxes; ++b)
        if (p->box_leaf[b] >= 0) leaf_box[p->box_leaf[b]] = b;
    for (int i = 0; i < d.n_leaves; ++i) {
        lcls[i] = p->tree.leaves[i].cls;
        llev[i] = p->tree.leaves[i].level;
        lix[i] = p->tree.leaves[i].ix;
        liy[i] = p->tree.leaves[i].iy;
    }
    d.leaf_box = dev_upload(leaf_box);
    d.leaf_cls = dev_upload(lcls);
    p->ext.leaf_level = dev_upload(llev);
    p->ext.leaf_ix = dev_upload(lix);
    p->ext.leaf_iy = dev_upload(liy);
    // interaction lists, built on the device once per geometry (per level)
    build_lists_device(p, s);
    setup_tables(p);
    // extension data
    const StencilInfo &st = p->st;
    DevExt &x = p->ext;
    x.ncut = (int)st.cut_leaf.size();
    x.cut_leaf = dev_upload(st.cut_leaf);
    x.n_interior = dev_upload(st.n_interior);
    x.grid_src = dev_upload(st.grid_src);
    x.node_src = dev_upload(st.node_src);
    x.stencil_off = dev_upload(st.stencil_off);
    x.pinv_off = dev_upload(st.pinv_off);
    x.reg_leaf_off = dev_upload(st.reg_leaf_off);
    x.owned_off = dev_upload(st.owned_off);
    x.owned = dev_upload(st.owned);
    x.pinv = dev_upload(st.pinv);
    const bool lines = st.mode == 1;   // extension along lines: no universal operator, line coefficients instead
    std::vector<double> Ag(lines ? 0 : (size_t)st.Kbar * st.Kbar * st.NG);
    for (int g = 0; !lines && g < st.Kbar * st.Kbar; ++g)
        std::copy(&st.A[(size_t)(p->KK + g) * st.NG], &st.A[(size_t)(p->KK + g) * st.NG] + st.NG, &Ag[(size_t)g * st.NG]);
    x.A_grid = dev_upload(Ag);
    x.mode = st.mode;
    x.n_ray = (int)st.ray_c.size();
    x.ray_c = dev_upload(st.ray_c);
    x.ray_g = dev_upload(st.ray_g);
    x.ray_src = dev_upload(st.ray_src);
    x.ray_coef = dev_upload(st.ray_coef);
    if (lines && p->opt.precision != VPX_PREC_MIXED)
        x.Fall = dev_alloc<double>((size_t)p->opt.max_rhs * x.ncut * st.Kbar * st.Kbar);
    x.cheb_inv = dev_upload(st.cheb_inv);
    if (p->opt.precision == VPX_PREC_MIXED) {
        // double-float copies for the mixed form's extension
        auto split = [](double v) {
            const float h = (float)v;
            return DevExt::DfPair{h, (float)(v - (double)h)};
        };
        // A_I^+ rows padded to an even length so that every row block is 16-byte aligned
        std::vector<int64_t> poff(st.cut_leaf.size(), 0);
        size_t tot = 0;
        for (size_t c = 0; !lines && c < st.cut_leaf.size(); ++c) {
            poff[c] = (int64_t)tot;
            tot += (size_t)st.NG * ((st.n_interior[c] + 1) & ~1);
        }
        // the Chebyshev transform padded to an even length (16-byte multiple) likewise
        std::vector<DevExt::DfPair> pd(tot, DevExt::DfPair{0.f, 0.f}), cd((st.cheb_inv.size() + 1) & ~(size_t)1,
                                                                           DevExt::DfPair{0.f, 0.f});
        for (size_t c = 0; !lines && c < st.cut_leaf.size(); ++c) {
            const int nI = st.n_interior[c], nIp = (nI + 1) & ~1;
            for (int k = 0; k < st.NG; ++k)
                for (int i = 0; i < nI; ++i)
                    pd[poff[c] + (size_t)k * nIp + i] = split(st.pinv[st.pinv_off[c] + (size_t)k * nI + i]);
        }
        for (size_t i = 0; i < st.cheb_inv.size(); ++i) cd[i] = split(st.cheb_inv[i]);
        x.pinv_df = dev_upload(pd);
        x.pinv_df_off = dev_upload(poff);
        x.cheb_df = dev_upload(cd);
        // A_{X_Sbar,G} c of every cut leaf as one table pass; targets of the Chebyshev stage
        const int Kb2 = st.Kbar * st.Kbar;
        if (x.ncut > 0 && !lines) {
            std::vector<std::pair<int, GPair>> tg;
            for (int c = 0; c < x.ncut; ++c) tg.push_back({0, GPair{c, 0, (int64_t)c * Kb2, 1.0}});
            gemm_pass_upload_tables(x.grid_pass, Ag, 1, Kb2, st.NG, true);
            x.grid_pass.add = 0;
            gemm_pass_set_pairs(x.grid_pass, tg);
        }
        std::vector<int32_t> tc, tl;
        for (int c = 0; c < x.ncut; ++c) {
            tc.push_back(c);
            tl.push_back(st.cut_leaf[c]);
        }
        for (int c = 0; c < x.ncut; ++c)
            for (int j = st.owned_off[c]; j < st.owned_off[c + 1]; ++j) {
                tc.push_back(c);
                tl.push_back(st.owned[j]);
            }
        x.n_tgt = (int)tc.size();
        x.tgt_cut = dev_upload(tc);
        x.tgt_leaf = dev_upload(tl);
        // target geometry in the coordinates of the cut leaf's Sbar (half side r):
        // z = offset + scale * t for the leaf nodes t on [-1, 1]
        std::vector<double> geo((size_t)4 * x.n_tgt);
        for (int t = 0; t < x.n_tgt; ++t) {
            const Leaf &S = p->tree.leaves[st.cut_leaf[tc[t]]], &T = p->tree.leaves[tl[t]];
            const double sS = std::ldexp(1.0, -S.level), sT = std::ldexp(1.0, -T.level), r = 1.5 * sS;
            const double cxS = -0.5 + (S.ix + 0.5) * sS, cyS = -0.5 + (S.iy + 0.5) * sS;
            const double cxT = -0.5 + (T.ix + 0.5) * sT, cyT = -0.5 + (T.iy + 0.5) * sT;
            geo[4 * t] = (cxT - cxS) / r;
            geo[4 * t + 1] = (cyT - cyS) / r;
            geo[4 * t + 2] = 0.5 * sT / r;
            geo[4 * t + 3] = (tl[t] == st.cut_leaf[tc[t]]) ? 1.0 : 0.0;
        }
        x.tgt_geo = dev_upload(geo);
        for (int c = 0; c < x.ncut; ++c) x.max_interior = std::max(x.max_interior, st.n_interior[c]);
        x.cbuf = dev_alloc<double>(lines ? 1 : (size_t)p->opt.max_rhs * x.ncut * st.NG);
        x.Fall = dev_alloc<double>((size_t)p->opt.max_rhs * x.ncut * Kb2);
        x.alpha = dev_alloc<DevExt::DfPair>((size_t)p->opt.max_rhs * x.ncut * ((Kb2 + 1) & ~1));
    }
    // boundary
    p->wk.bdry_leaf = dev_upload(p->bdry_leaf);
    p->wk.bdry_w = dev_upload(p->bdry_w);
    // workspace
    DevWork &w = p->wk;
    w.max_rhs = p->opt.max_rhs;
    w.fe = dev_alloc<double>((size_t)w.max_rhs * d.n_leaves * p->KK);
    w.mpole = dev_alloc<double>((size_t)w.max_rhs * d.n_boxes * 2 * p->P);
    w.local = dev_alloc<double>((size_t)w.max_rhs * d.n_boxes * 2 * p->P);
    w.status = dev_alloc<int>(1);
    w.charge_part = dev_alloc<double>((size_t)w.max_rhs * charge_blocks(d.n_leaves));
    x.grid_pass.status = w.status;
    VPX_CUDA(cudaMemset(w.status, 0, sizeof(int)));
    setup_near_pairs(p);
    setup_passes(p);
    VPX_CUDA(cudaDeviceSynchronize());
}

void device_copy_near_tables(vpx_plan *p, double *out) {
    VPX_CUDA(cudaMemcpy(out, p->tab.near, sizeof(double) * kNearConfigs * p->KK * p->KK, cudaMemcpyDeviceToHost));
}

void device_free(vpx_plan *p) {
    device_bie_free(p);
    DevTree &d = p->dt;
    dev_free(d.box_level); dev_free(d.box_ix); dev_free(d.box_iy); dev_free(d.box_parent);
    dev_free(d.box_child0); dev_free(d.box_leaf); dev_free(d.box_morton); dev_free(d.box_nz);
    dev_free(d.leaf_box); dev_free(d.leaf_cls); dev_free(d.leaf_nz);
    dev_free(d.near); dev_free(d.vlist); dev_free(d.xlist); dev_free(d.wlist);
    DevTables &t = p->tab;
    dev_free(t.near); dev_free(t.w2); dev_free(t.s2l); dev_free(t.bary); dev_free(t.tnodes);
    DevExt &x = p->ext;
    dev_free(x.cut_leaf); dev_free(x.n_interior); dev_free(x.grid_src); dev_free(x.node_src);
    dev_free(x.stencil_off); dev_free(x.pinv_off); dev_free(x.reg_leaf_off); dev_free(x.owned_off);
    dev_free(x.owned); dev_free(x.pinv); dev_free(x.A_grid); dev_free(x.cheb_inv);
    dev_free(x.pinv_df); dev_free(x.cheb_df); dev_free(x.pinv_df_off); dev_free(x.tgt_geo);
    gemm_pass_free(x.grid_pass);
    dev_free(x.tgt_cut); dev_free(x.tgt_leaf); dev_free(x.cbuf); dev_free(x.Fall); dev_free(x.alpha);
    dev_free(x.ray_c); dev_free(x.ray_g); dev_free(x.ray_src); dev_free(x.ray_coef);
    dev_free(x.leaf_level); dev_free(x.leaf_ix); dev_free(x.leaf_iy); dev_free(x.owned_flag_dev);
    free_passes(p);
    DevWork &w = p->wk;
    dev_free(w.fe); dev_free(w.mpole); dev_free(w.local);
    dev_free(w.nz_leaves); dev_free(w.bdry_leaf); dev_free(w.bdry_w); dev_free(w.status);
    dev_free(w.f_tmp); dev_free(w.v_tmp); dev_free(w.b_tmp); dev_free(w.charge_part);
    for (auto &ev : p->events)
        if (ev) {
            cudaEventDestroy((cudaEvent_t)ev);
            ev = nullptr;
        }
    if (p->graph_exec) {
        cudaGraphExecDestroy((cudaGraphExec_t)p->graph_exec);
        p->graph_exec = nullptr;
    }
    for (void **e : {&p->ev_fork, &p->ev_up, &p->ev_join, &p->ev_join2, &p->ev_lc, &p->ev_lvf, &p->ev_lv,
                     &p->ev_bfork, &p->ev_bjoin})
        if (*e) {
            cudaEventDestroy((cudaEvent_t)*e);
            *e = nullptr;
        }
    for (void **st : {&p->aux_stream, &p->aux2_stream})
        if (*st) {
            cudaStreamDestroy((cudaStream_t)*st);
            *st = nullptr;
        }
    if (p->stream) {
        cudaStreamDestroy((cudaStream_t)p->stream);
        p->stream = nullptr;
    }
}

}  // namespace vpx
