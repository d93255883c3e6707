// ext.cuh -- arguments of the extension kernels (Sections 3.2, 4.1): the FP64
// kernel (device_exec.cu) and the double-float one of the mixed form
// (extend_df.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace vpx {

// an extension target in the coordinates of its cut leaf's Sbar: node
// coordinate z = (ox or oy) + sc * t for the leaf nodes t on [-1, 1]
struct ExtTgtGeo {
    double ox, oy, sc, self;   // self: 1 for the cut leaf itself
};

struct ExtArgs {
    int K, Kbar, NG;
    const int32_t *cut_leaf, *n_interior, *grid_src, *node_src, *owned_off, *owned;
    const int64_t *stencil_off, *pinv_off;
    const double *pinv, *A_grid, *cheb_inv, *tnodes;
    const float2 *pinv_df;      // P_S as double-float (hi, lo), rows padded to an even length
    const int64_t *pinv_df_off; // start of each cut leaf's P_S in pinv_df (even)
    const float2 *cheb_df;      // [Kbar][Kbar] double-float
    const int32_t *leaf_level, *leaf_ix, *leaf_iy;
    const double *f;
    int64_t ldf;
    double *fe;
    int64_t ldfe;
    // extension along lines: the exterior grid values, [rhs][cut][Kbar^2] (null: universal stencil)
    const double *ray_F = nullptr;
    int64_t ldR = 0;
    // mixed form: the exact bf16 slices of the leaf values written with them,
    // [rhs][n_leaves][kSlicesS][kpad] and exponents [rhs][n_leaves] (null: not sliced here)
    uint16_t *fe_sl = nullptr;
    int32_t *fe_ex = nullptr;
    int n_leaves = 0, kpad = 0;
};

// mixed form (extend_df.cu): c = A_I^+ f_I into cbuf[rhs][cut][NG]; then, after
// the grid values A_{X_Sbar,G} c are in Fall[rhs][cut][Kbar^2], the Chebyshev
// stage for every target leaf (tgt_cut[t], tgt_leaf[t])
void extend_df_prepare(int max_interior, int K, int Kbar);
void launch_ext_coeff_df(const ExtArgs &a, int ncut, int max_interior, int nrhs, double *cbuf, int64_t ldc,
                         int *status, cudaStream_t s);
void launch_ext_eval_df(const ExtArgs &a, int ncut, int n_tgt, const int32_t *tgt_cut, const int32_t *tgt_leaf,
                        const ExtTgtGeo *geo, const double *Fall, int64_t ldF, float2 *alpha, int nrhs, int *status,
                        cudaStream_t s);

}  // namespace vpx
