// internal.h -- private declarations of the vpx library (host + device).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vpx.h"

namespace vpx {

constexpr int kMaxLevel = 15;     // ix, iy < 2^15
constexpr int kMaxK = 16;
constexpr int kMaxP = 64;         // expansion terms (p + 1)
constexpr int kNearConfigs = 33;  // 9 colleagues + 12 coarse + 12 fine (Section 4, Fig. tree_levels)
constexpr int kVSlots = 40;       // list i offsets: [-3,3]^2 minus [-1,1]^2
constexpr int kXSlots = 20;       // list i+ (coarse leaf) relative positions
constexpr int kWSlots = 20;       // list i- (fine box) relative positions
constexpr double kPi = 3.14159265358979323846;

enum LeafClass : int32_t { kRegular = 0, kCut = 1, kExterior = 2 };

// ------------------------------------------------------------------ errors
struct Error {
    int code;
    std::string msg;
};
void set_error_message(const std::string &m);
[[noreturn]] void fail(int code, const std::string &m);

// ------------------------------------------------------------- quadrature
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);   // [-1,1], ascending
void gauss_log_rule(int n, std::vector<double> &x, std::vector<double> &w);   // weight -r log r on [0,1]
std::vector<double> chebyshev1(int n);                                        // ascending
void padua(int q, std::vector<double> &x, std::vector<double> &y);
std::vector<double> barycentric_weights(const std::vector<double> &t);
void lagrange_eval(const std::vector<double> &t, const std::vector<double> &bw, double s, double *out);

// ------------------------------------------------------------- box keys
inline uint64_t box_key(int level, int ix, int iy) {
    return (uint64_t(level) << 56) | (uint64_t(uint32_t(ix)) << 28) | uint64_t(uint32_t(iy));
}
inline int key_level(uint64_t k) { return int(k >> 56); }
inline int key_ix(uint64_t k) { return int((k >> 28) & 0xFFFFFFF); }
inline int key_iy(uint64_t k) { return int(k & 0xFFFFFFF); }
uint32_t morton2(uint32_t ix, uint32_t iy);   // x in even bits, y in odd bits

struct Leaf {
    int32_t level, ix, iy, cls, owner;
};

// The tree as the host builds it.
struct HostTree {
    int K = 0;
    std::vector<Leaf> leaves;            // Z-order
    int max_level = 0;
};

struct Callbacks {
    vpx_curve_cb curve;
    vpx_inside_cb inside;
    vpx_points_cb f;
    void *ctx;
    int n_panels;
};

void build_tree(const vpx_options &opt, const Callbacks &cb, HostTree &tree);

// ------------------------------------------------------- boundary correction
// Host part of the interior Dirichlet correction (Section 5): Nystrom
// geometry and, per leaf node within reach of a panel, the product-integration
// weights that replace that panel's Gauss-Legendre terms.
struct BieDev {                          // device copies (device plans only)
    double *y = nullptr, *nu = nullptr, *sw = nullptr, *leaf_xy = nullptr, *corr_w = nullptr, *log_c = nullptr;
    int64_t *corr_off = nullptr;
    int32_t *corr_panel = nullptr;
    double *rhs = nullptr, *cst = nullptr;
    double *minv = nullptr;              // [n_unknowns][n_unknowns] inverse of the Nystrom system
};

struct BieHost {
    bool ready = false;
    int n_log = 0, n_unknowns = 0;         // log terms; N + n_log
    std::vector<int32_t> log_curve;        // curve of each log term (the holes, or every inclusion)
    std::vector<double> log_centre;        // a point inside that curve, 2 per term
    BieDev dev;
    int nq = 0, n_panels = 0, n_curves = 0, outer_curve = -1;   // outer_curve -1: an exterior problem
    std::vector<double> nu, sw, kappa;     // outward normal (2 per node), s*w, signed curvature
    std::vector<int32_t> curve_of_node;    // closed curve of every boundary node
    std::vector<double> jump;              // -1/2 on the outer curve, +1/2 on curves Omega surrounds
    std::vector<int64_t> corr_off;         // [n_leaf_nodes + 1]
    std::vector<int32_t> corr_panel;       // panel of each correction
    std::vector<double> corr_w;            // [n_corr][nq]: product weight minus the plain term
    std::vector<double> p2m;               // [N][2P]: each node's dipole (sigma = 1) as a multipole of its leaf
};

// ------------------------------------------------------- stencil / extension
struct StencilInfo {
    int q = 0, Kbar = 0, NG = 0, NX = 0;       // NX = K*K + Kbar*Kbar + NG universal points
    std::vector<double> ref_xy;                // NX universal points on [-1,1]^2 of Sbar (X_S, X_Sbar, G)
    std::vector<double> A;                     // NX x NG universal matrix (row-major): Lagrange basis of P_q at G
    std::vector<double> cheb_inv;              // Kbar x Kbar: alpha_m = sum_a C[m][a] F_a
    // per cut leaf
    std::vector<int32_t> cut_leaf;             // leaf index
    std::vector<int64_t> stencil_off;          // offset of its block in the f column
    std::vector<int32_t> n_interior;           // N_I
    std::vector<int64_t> pinv_off;             // offset of P_S (NG x N_I, row-major)
    std::vector<double> pinv;                  // all P_S
    std::vector<int32_t> grid_src;             // [ncut][Kbar^2]: index into the block, -1 exterior
    std::vector<int32_t> node_src;             // [ncut][K^2]: index into the block, -1 exterior node
    std::vector<int32_t> owned_off, owned;     // CSR: owned exterior leaves per cut leaf
    std::vector<int64_t> reg_leaf_off;         // [n_leaves] stencil offset of a regular leaf, -1 otherwise
    double max_pinv_norm = 0.0, max_cond = 0.0;
    // extension along lines (mode 1): per exterior grid point of every cut leaf
    int mode = 0;
    std::vector<int32_t> ray_c, ray_g;         // cut leaf, grid index (by*Kbar + ax)
    std::vector<int64_t> ray_src;              // position of its first line point in the f column
    std::vector<double> ray_coef;              // [n][8]: Floater-Hormann coefficients of its line points
};

// The universal operator of leaf order K on [-1,1]^2 (rows X_S, X_Sbar, G),
// flat limit plus (rbf_eps / 2)^2 A2 for rbf_eps > 0.
void universal_operator(int K, double rbf_eps, std::vector<double> &A, int &NX, int &NG);
// A2 of the Gaussian operator for leaf order K (rbf_eps2_tables.cpp); false if K has no table.
bool rbf_eps2_table(int K, const double **a2, int *nx, int *ng);
// rbf_eps in [0, 1e-3], and a table for K when positive; else VPX_ERR_ARG.
void check_rbf_eps(int K, double rbf_eps);
void build_stencil(const vpx_options &opt, const Callbacks &cb, const HostTree &tree,
                   std::vector<double> &stencil_xy, StencilInfo &st, bool compute_operators);

}  // namespace vpx
