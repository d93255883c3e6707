// gemm.cuh -- grouped "table x gathered vectors" GEMM, the one shape every
// contraction of the hot path takes:
//
//   out[dst_p + i] (+)= scale_p * sum_k Tab_{t(p)}[i][k] * vec_{src_p}[k]
//
// for every pair p of a pass; pairs are grouped by table into tiles of at most
// 64 pairs.  Near field (33 tables), L2M (1), M2M (4), M2L (40), S2L (20),
// L2L (4), L2T (1) and M2T (20) are all passes of this form.  Two engines run
// it: FP64 register tiles (the FP64 form) and exact bf16 slices on the tensor
// cores with FP64 recombination (the mixed form, see gemm.cu).
#pragma once

#include <cstdint>
#include <vector>

namespace vpx {

constexpr int kGemmTileN = 64;   // pairs per tile (FP64 engine)
constexpr int kWsTileN = 48;     // pairs per tile (tcgen05 engine)
constexpr int kFragBigPass = 4096;   // fragment engine: 32 pairs per tile from this many pairs on, else 8
constexpr int kRowsTileN = 1;        // pairs per tile (double-float row engine)
constexpr int kSlicesS = 5;      // bf16 slices per operand in the mixed form (39 bits); the int64
                                 // recombination holds 2^24 * 256^4
constexpr int kSliceBitsB = 8;   // bits per slice: balanced base-256 digits, |digit| <= 128

struct GPair {
    int32_t src;      // source vector index
    int32_t pad;
    int64_t dst;      // output offset (elements) within one right-hand side
    double scale;
};

struct GTile {
    int32_t tab, first, count, pad;
};

struct VecSet {                        // source vectors of a pass
    const double *base = nullptr;      // vector v of rhs r at base + r*ld + v*stride
    int64_t ld = 0;
    int stride = 0;
    uint16_t *slices = nullptr;        // mixed form: [rhs][nvec][S][Kpad], or null: sliced where used
    int32_t *expo = nullptr;           // [rhs][nvec]
    int nvec = 0;
    int kpad = 0;                      // inner length of the stored slices
};

// One pass on the device.
struct GemmPass {
    int M = 0, Kd = 0, Kpad = 0, Mpad = 0, ntab = 0;
    int add = 1;                       // 1: atomic add into out, 0: store
    int *status = nullptr;             // device status word (bounded waits report here)
    const double *tab = nullptr;       // [ntab][M][Kd] FP64 (row-major)
    const uint16_t *tslices = nullptr; // [ntab][S][Mpad][Kpad] bf16 bits (mixed form)
    const int32_t *texpo = nullptr;    // [ntab][Mpad] row exponents (mixed form)
    const uint32_t *tfrag = nullptr;   // [ntab][S][Mpad/16][Kpad/16][32 lanes][4] mma.sync A fragments (mixed form)
    GPair *pairs = nullptr;
    GTile *tiles = nullptr;            // kGemmTileN pairs each
    GTile *tiles_f = nullptr;          // np_f pairs each (fragment engine)
    GTile *tiles_r = nullptr;          // kRowsTileN pairs each (row engine)
    GTile *tiles_w = nullptr;          // kWsTileN pairs each (tcgen05 engine)
    const void *tdfT = nullptr;        // [ntab][Kd][M] double-float (float hi, lo): the row engine runs the pass
    const uint16_t *tint = nullptr;    // [ntab][S][Kpad/8][Mpad][8] slices, column chunks interleaved (tcgen05 engine)
    int ws_kind = 0;                   // 0: not on that engine; 1: on it (table rows on M)
    int n_pairs = 0, n_tiles = 0, n_tiles_f = 0, np_f = 8, n_tiles_r = 0, n_tiles_w = 0;
    // the fragment engine's other tile width (8 <-> 32 pairs), for the autotuner
    GTile *tiles_f_alt = nullptr;
    int n_tiles_f_alt = 0, np_f_alt = 32;
    int engine = 0;                    // 0: default routing; 1: fragment engine even where tcgen05 is eligible
    bool owns_tables = true;           // false: a view of another pass's tables (gemm_pass_view)
    std::vector<GPair> h_pairs;        // host copy (setup)
};

// The schedule choices of one mixed-form pass that the autotuner may change.
struct GemmChoice {
    int engine;   // 0: default routing (tcgen05 where eligible), 1: fragment engine
    int np_f;     // fragment-engine pairs per tile (8 or 32; 0: keep the current width)
};
GemmChoice gemm_choice(const GemmPass &g);
void gemm_set_choice(GemmPass &g, GemmChoice c);

// One recorded call of gemm_run (the autotuner replays recorded calls).
struct GemmCall {
    GemmPass *g;
    VecSet vs;
    double *out;
    int64_t ldo;
    int nrhs;
};
// While non-null, gemm_run appends every mixed-form call it makes on this thread.
void gemm_set_recorder(std::vector<GemmCall> *rec);

// Host helpers
// (table, pair); frag_np: pairs per fragment-engine tile (8 or 32; 0: by pass size)
void gemm_pass_set_pairs(GemmPass &g, std::vector<std::pair<int, GPair>> &tagged, int frag_np = 0);
void gemm_pass_upload_tables(GemmPass &g, const std::vector<double> &tab, int ntab, int M, int Kd, bool mixed);
void gemm_pass_free(GemmPass &g);
// v takes base's tables (shared, not copied: base must outlive v) and routing;
// its pairs are set afterwards with gemm_pass_set_pairs
void gemm_pass_view(GemmPass &v, const GemmPass &base);
// Hand a mixed-form pass to the double-float row engine (gemm_rows.cu) when
// its rows fit one CTA and every pair scale is a power of two; returns whether.
bool gemm_pass_use_rows(GemmPass &g, const std::vector<double> &tab);
// fragment engine (gemm_frag.cu)
void gemm_frag_prepare_device();
// warp-specialised tcgen05 engine (gemm_ws.cu): interleaved table copy of a mixed-form pass
void gemm_ws_prepare(GemmPass &g);
void gemm_ws_prepare_device();


// Launches (stream s): run a pass on nrhs right-hand sides.
void gemm_run(const GemmPass &g, const VecSet &vs, double *out, int64_t ldo, int nrhs, bool mixed, void *s);
// Slice vectors [first, first+count) of a set (mixed form), per rhs.
void slice_vectors(const VecSet &vs, int first, int count, int Kd, int Kpad, int nrhs, void *s);

}  // namespace vpx
