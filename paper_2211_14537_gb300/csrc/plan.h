// plan.h -- the plan object behind vpx_plan_t (host + device state).
#pragma once

#include <cstdint>
#include <vector>

#include "gemm.cuh"
#include "internal.h"

struct vpx_plan;

namespace vpx {

// Device-resident tree and lists (raw device pointers).
struct DevTree {
    int n_leaves = 0, n_boxes = 0, n_levels = 0;
    int32_t level_start[kMaxLevel + 2] = {0};
    int32_t *box_level = nullptr, *box_ix = nullptr, *box_iy = nullptr, *box_parent = nullptr;
    int32_t *box_child0 = nullptr, *box_leaf = nullptr;
    uint32_t *box_morton = nullptr;     // Morton key within its level (sorted per level)
    uint8_t *box_nz = nullptr;          // subtree carries a non-zero source
    int32_t *leaf_box = nullptr, *leaf_cls = nullptr;
    uint8_t *leaf_nz = nullptr;
    // fixed-slot interaction lists (-1 = empty)
    int32_t *near = nullptr;   // [n_leaves][33]  source leaf per near-field configuration
    int32_t *vlist = nullptr;  // [n_boxes][40]   source box per list-i offset
    int32_t *xlist = nullptr;  // [n_boxes][20]   source leaf per list-i+ configuration
    int32_t *wlist = nullptr;  // [n_leaves][20]  source box per list-i- position
};

struct DevTables {
    double *near = nullptr;     // [33][KK][KK]
    double *w2 = nullptr;       // [KK] tensor Gauss-Legendre weights on [-1,1]^2
    double *s2l = nullptr;      // [20][KK][P] complex
    double *bary = nullptr;     // [K] barycentric weights of the leaf nodes
    double *tnodes = nullptr;   // [K] leaf nodes on [-1,1]
};

struct DevExt {
    int ncut = 0;
    int32_t *cut_leaf = nullptr, *n_interior = nullptr, *grid_src = nullptr, *node_src = nullptr;
    int64_t *stencil_off = nullptr, *pinv_off = nullptr, *reg_leaf_off = nullptr;
    int32_t *owned_off = nullptr, *owned = nullptr;
    double *pinv = nullptr;       // all P_S
    double *A_grid = nullptr;     // [Kbar^2][NG] rows of the universal A at X_Sbar
    double *cheb_inv = nullptr;   // [Kbar][Kbar]
    // double-float copies (hi, lo float pairs) for the mixed form
    struct DfPair { float hi, lo; };
    DfPair *pinv_df = nullptr, *cheb_df = nullptr;   // pinv_df: rows padded to an even length
    int64_t *pinv_df_off = nullptr;
    double *tgt_geo = nullptr;                         // [n_tgt][4]: offset x, offset y, node scale, is-cut-leaf
    GemmPass grid_pass;                  // A_{X_Sbar,G} c for all cut leaves (one table)
    int n_tgt = 0, max_interior = 0;
    int32_t *tgt_cut = nullptr, *tgt_leaf = nullptr;   // extension targets: cut leaves, then their lists
    double *cbuf = nullptr, *Fall = nullptr;           // [max_rhs][ncut][NG], [max_rhs][ncut][Kbar^2]
    DfPair *alpha = nullptr;                           // [max_rhs][ncut][Kbar^2 rounded up to even] truncated Chebyshev coefficients
    int32_t *leaf_level = nullptr, *leaf_ix = nullptr, *leaf_iy = nullptr;
    int32_t *owned_flag_dev = nullptr;   // [n_leaves] 1 if the leaf is in an extension list
    // extension along lines: exterior grid points and their line-point coefficients
    int mode = 0, n_ray = 0;
    int32_t *ray_c = nullptr, *ray_g = nullptr;
    int64_t *ray_src = nullptr;
    double *ray_coef = nullptr;
};

struct DevWork {
    int max_rhs = 0;
    double *fe = nullptr;         // [max_rhs][n_leaves][KK]
    double *mpole = nullptr;      // [max_rhs][n_boxes][2P]
    double *local = nullptr;      // [max_rhs][n_boxes][2P]
    int32_t *nz_leaves = nullptr; // leaves with non-zero source
    int n_nz_leaves = 0;
    int32_t *bdry_leaf = nullptr; // [n_bdry]
    double *bdry_w = nullptr;     // [n_bdry][2K] Lagrange weights (x then y)
    int *status = nullptr;        // device status word
    double *f_tmp = nullptr, *v_tmp = nullptr, *b_tmp = nullptr;   // for vpx_execute_host
    double *charge_part = nullptr;    // [max_rhs][charge_blocks(n_leaves)] block sums of the net charge
};

// Blocks of the net-charge reduction (8 leaves per block, at most two per SM's worth of 152 SMs).
inline int charge_blocks(int n_leaves) {
    const int b = (n_leaves + 7) / 8;
    return b < 1 ? 1 : (b > 304 ? 304 : b);
}

// The level chains (M2M up, L2L down) as one persistent launch each (chain.cu).
struct ChainPlan {
    bool ok = false;              // false: the per-level passes run the chains
    int n_up = 0, n0_up = 0, n_down = 0, n0_down = 0, max_ctas = 0;
    void *tab_up = nullptr, *tab_down = nullptr;     // [4][P][P] complex tables (FP64 or hi/lo float pairs)
    int16_t *kr_up = nullptr, *kr_down = nullptr;     // [4][P][2] non-zero column ranges
    int32_t *items_up = nullptr, *items_down = nullptr, *need = nullptr;
    int32_t *up_of = nullptr;     // per box: parent, position among its siblings (pairs)
    int *ws = nullptr;            // both queue blocks, zeroed before every step
    size_t ws_ints = 0;
    // mixed form: the warp-granular kernel's packed rows (double-float complex) and row starts
    void *tabw_up = nullptr, *tabw_down = nullptr;
    int32_t *roff_up = nullptr, *roff_down = nullptr;
    int np_up = 0, np_down = 0, max_ctas_w = 0;
    size_t smem_w = 0;
};

struct FmmPasses {                // every contraction of the box FMM as a grouped table GEMM
    GemmPass l2m, m2l, s2l, l2t, m2t, near;
    // the level chains in bands of levels (one launch each, views of the
    // composed tables in m2m_tab / l2l_tab): upward bands from the deepest
    // level, a first downward launch (l2l_pre), then downward bands
    GemmPass m2m[kMaxLevel + 1], l2l[kMaxLevel + 1], l2l_pre, m2m_tab, l2l_tab;
    int n_m2m = 0, n_l2l = 0;
    uint16_t *fe_sl = nullptr, *mp_sl = nullptr;   // exact bf16 slices of leaf values, multipoles (mixed form)
    // gather lists of the constant terms: boxes from lc_first on (locals), leaves (potentials)
    int lc_first = 0, lc_rows = 0;
    int32_t *lc_off = nullptr, *lc_idx = nullptr, *tc_off = nullptr, *tc_idx = nullptr;
    double *lc_coef = nullptr, *tc_coef = nullptr;
    int32_t *fe_ex = nullptr, *mp_ex = nullptr;
    ChainPlan chain;
};

}  // namespace vpx

struct vpx_plan {
    uint64_t uid = 0;             // unique per plan of the process (keys of cached batch graphs)
    int64_t tune_epoch = 0;       // bumped whenever the autotuner changes a pass (keys of cached graphs)
    vpx_options opt{};
    bool host_only = false;
    int K = 0, KK = 0, P = 0;
    vpx::HostTree tree;
    vpx::StencilInfo st;
    std::vector<double> stencil_xy;
    std::vector<double> leaf_xy;
    std::vector<double> bdry_xy;
    std::vector<int32_t> bdry_leaf;
    std::vector<double> bdry_w;
    std::vector<double> bdry_dxy;     // gamma_i'(t_j) at the boundary nodes
    std::vector<double> bdry_ends;    // per panel gamma_i(-1), gamma_i(1): 4 doubles
    vpx::BieHost bie;                 // boundary correction (host part), filled by vpx_bie_setup
    // host copies of the boxes (level, Morton order) and lists
    std::vector<int32_t> box_level, box_ix, box_iy, box_parent, box_child0, box_leaf;
    std::vector<uint32_t> box_morton;
    std::vector<uint8_t> box_nz, leaf_nz;
    std::vector<int32_t> near, vlist, xlist, wlist;
    int32_t level_start[vpx::kMaxLevel + 2] = {0};
    int n_levels = 0;
    int64_t cnt_near = 0, cnt_m2l = 0, cnt_s2l = 0, cnt_m2t = 0;
    // device
    int device = -1;
    void *stream = nullptr;       // plan-owned stream for vpx_execute_host
    void *last_stream = nullptr;
    vpx::DevTree dt;
    vpx::DevTables tab;
    vpx::DevExt ext;
    vpx::DevWork wk;
    vpx::FmmPasses fmm;
    bool timing = false;
    void *events[VPX_N_PASSES + 3] = {nullptr};   // pass boundaries on the main stream, near field on aux
    void *aux_stream = nullptr;   // second stream of the execute graph (near field)
    void *aux2_stream = nullptr;  // third stream (lists i+ and i-)
    int64_t graph_kernels = 0;    // kernel nodes of the captured execute graph
    void *ev_fork = nullptr, *ev_up = nullptr, *ev_join = nullptr, *ev_join2 = nullptr;
    void *ev_lc = nullptr;    // list i+ and the local constant terms done (third stream)
    void *ev_lvf = nullptr, *ev_lv = nullptr;   // leaf values beside the extension: fork / done
    void *ev_bfork = nullptr, *ev_bjoin = nullptr;   // batch fork / join on the plan's own stream
    void *graph_exec = nullptr;   // captured vpx_execute sequence (cudaGraphExec_t)
    int64_t graph_key[10] = {0};
    double pass_ms[VPX_N_PASSES] = {0};
};

namespace vpx {
// host list builder (same routine the device kernel runs)
void build_boxes(vpx_plan *p);
void build_lists_host(vpx_plan *p);
// device side (device.cu)
void device_setup(vpx_plan *p);
void device_free(vpx_plan *p);
void device_extend(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *fe_out, int64_t ldfe, void *stream);
void device_potential(vpx_plan *p, const double *fe_in, int64_t ldfe, int nrhs, double *v, int64_t ldv,
                      double *vb, int64_t ldb, void *stream);
void device_execute(vpx_plan *p, const double *f, int nrhs, int64_t ldf, double *v, int64_t ldv, double *vb,
                    int64_t ldb, void *stream);
int device_sync_status(vpx_plan *p);
int device_check_bounded_wait(int *status_out);   // selftest.cu
void device_execute_batch(int n, vpx_plan *const *plans, const double *const *f, const int *nrhs, const int64_t *ldf,
                          double *const *v, const int64_t *ldv, double *const *vb, const int64_t *ldb, void *stream);
void device_copy_near_tables(vpx_plan *p, double *out);
void device_autotune(int n, vpx_plan *const *plans, const double *const *f, const int *nrhs, const int64_t *ldf,
                     void *stream, int *n_passes, int *n_changed);
void device_potential_static(vpx_plan *p, const double *fe_in, int64_t ldfe, int nrhs, double *v, int64_t ldv,
                             double *vb, int64_t ldb, void *stream);
void device_execute_host(vpx_plan *p, const double *f, int nrhs, double *v, double *vb);
void device_net_charge(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *charge, void *stream);
void bie_setup(vpx_plan *p, vpx_inside_cb inside, void *ctx);
void device_bie_setup(vpx_plan *p);
void device_bie_solve(vpx_plan *p, const double *g, const double *vb, double growth, double *sol, void *stream);
void device_bie_eval(vpx_plan *p, const double *sol, const double *v, double *u, void *stream);
void device_bie_free(vpx_plan *p);
int gauss_jordan_inverse(int n, double *aug_dev, double *inv_dev);   // bie_device.cu
int device_check_gauss_jordan(int n, const double *a_host, double *inv_host);
}  // namespace vpx
