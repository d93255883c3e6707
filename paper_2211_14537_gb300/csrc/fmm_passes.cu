// fmm_passes.cu -- the box FMM (Section 4.1 with the lists of Fig. tree_levels)
// as a sequence of grouped table GEMMs (gemm.cuh), in the FP64 form or the
// exact-slice mixed form.
//
// Expansions of a box of side L and centre c (complex arithmetic written in
// real 2(p+1)-vectors, entries 2l, 2l+1 = Re, Im):
//   multipole  Phi(z) = a_0 log(z - c) + sum_{k>=1} at_k (L / (z - c))^k
//   local      Psi(z) = sum_{l>=0} bt_l ((z - c) / L)^l
// In these scaled variables every translation operator is independent of the
// level except for one real term a_0 log(L) (M2L, list i- evaluation) or
// a_0 log(H) (S2L, near field), which two small kernels add.
//
// Passes of one right-hand side (all pairs of a pass in one launch):
//   L2M (1 table)   leaf values        -> multipole of the leaf box (store)
//   M2M (4 tables)  child multipoles   -> parent multipole, level by level
//   M2L (40 tables) list-i multipoles  -> local             (all levels at once)
//   S2L (20 tables) list-i+ leaf values -> local
//   L2L (4 tables)  parent local       -> child local, level by level
//   L2T (1 table)   local              -> V at the K^2 nodes
//   M2T (20 tables) list-i- multipoles -> V at the K^2 nodes
//   near (33 tables) leaf values       -> V (tables of Section 4, Remark)
#include <cmath>
#include <complex>
#include <cstdlib>

#include "dev_common.cuh"
#include "gemm.cuh"

namespace vpx {

typedef std::complex<double> cd;

// ------------------------------------------------------- constant terms

// The level-dependent real terms of the scaled expansions, as fixed gather
// lists built at setup (row r: entries off[r] .. off[r+1] of (idx, coef)):
//   local[b][0] += log(L_b) sum_{list i} a_0(src) + sum_{list i+} log(H_src) a_0(src)
//   V[t][i]     += (1/2pi) [sum_near log(h_s) a_0(s) + sum_{list i-} log(L_W) a_0(W)]  (all i)
// with log(2^-l) = -l ln 2 folded into coef.  One warp per row.
__global__ void k_const_gather(int rows, int first, int P, const int32_t *off, const int32_t *idx,
                               const double *coef, const double *mpole, int64_t ldm, double *out, int64_t ldo,
                               int stride, int width) {
    pdl_entry();
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31, rhs = blockIdx.y;
    if (r >= rows) return;
    const double *mp = mpole + rhs * ldm;
    const int e0 = off[r], e1 = off[r + 1];
    double c = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) c += coef[e] * mp[(int64_t)idx[e] * 2 * P];
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    // atomic: the locals take M2L at the same time, V the near field and L2T
    double *o = out + rhs * ldo + (int64_t)(first + r) * stride;
    for (int i = lane; i < width; i += 32) atomicAdd(o + i, c);
}

// ------------------------------------------------------------ tables

static void real_form(const std::vector<cd> &C, int P, std::vector<double> &out, size_t off) {
    // C[row l][col k] complex (P x P) -> real 2P x 2P acting on (Re, Im) interleaved vectors
    for (int l = 0; l < P; ++l)
        for (int k = 0; k < P; ++k) {
            cd c = C[(size_t)l * P + k];
            out[off + (size_t)(2 * l) * 2 * P + 2 * k] = c.real();
            out[off + (size_t)(2 * l) * 2 * P + 2 * k + 1] = -c.imag();
            out[off + (size_t)(2 * l + 1) * 2 * P + 2 * k] = c.imag();
            out[off + (size_t)(2 * l + 1) * 2 * P + 2 * k + 1] = c.real();
        }
}

static std::vector<double> binom_table(int n) {
    std::vector<double> C((size_t)(n + 1) * (n + 1), 0.0);
    for (int i = 0; i <= n; ++i) {
        C[(size_t)i * (n + 1)] = 1.0;
        for (int j = 1; j <= i; ++j)
            C[(size_t)i * (n + 1) + j] = C[(size_t)(i - 1) * (n + 1) + j - 1] + (j < i ? C[(size_t)(i - 1) * (n + 1) + j] : 0.0);
    }
    return C;
}

void fmm_tables_host(vpx_plan *p, std::vector<double> &l2m, std::vector<double> &l2t, std::vector<double> &m2m,
                     std::vector<double> &l2l, std::vector<double> &m2l, std::vector<double> &m2t) {
    const int K = p->K, KK = p->KK, P = p->P, P2 = 2 * P;
    std::vector<double> t, tw;
    gauss_legendre(K, t, tw);
    std::vector<double> bw = barycentric_weights(t);
    // L2M: row 0 = weights; rows 2k, 2k+1 = Re, Im of -(1/k) 2^-k int l_j eta^k
    int nq = (K + P) / 2 + 2;
    std::vector<double> g, gw;
    gauss_legendre(nq, g, gw);
    std::vector<double> L((size_t)nq * K);
    for (int i = 0; i < nq; ++i) lagrange_eval(t, bw, g[i], &L[(size_t)i * K]);
    l2m.assign((size_t)P2 * KK, 0.0);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a) l2m[b * K + a] = tw[a] * tw[b];
    std::vector<cd> acc((size_t)P * KK, cd(0, 0));
    for (int i = 0; i < nq; ++i)
        for (int i2 = 0; i2 < nq; ++i2) {
            cd eta(g[i], g[i2]), pw(1.0, 0.0);
            double w = gw[i] * gw[i2];
            for (int k = 1; k < P; ++k) {
                pw *= eta * 0.5;
                cd c = -pw * (w / k);
                for (int b = 0; b < K; ++b)
                    for (int a = 0; a < K; ++a) acc[(size_t)k * KK + b * K + a] += c * (L[(size_t)i * K + a] * L[(size_t)i2 * K + b]);
            }
        }
    for (int k = 1; k < P; ++k)
        for (int j = 0; j < KK; ++j) {
            l2m[(size_t)(2 * k) * KK + j] = acc[(size_t)k * KK + j].real();
            l2m[(size_t)(2 * k + 1) * KK + j] = acc[(size_t)k * KK + j].imag();
        }
    // L2T: row i = target node: (Re xi^l, -Im xi^l), xi = (t_a + i t_b) / 2
    l2t.assign((size_t)KK * P2, 0.0);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a) {
            cd xi(0.5 * t[a], 0.5 * t[b]), pw(1.0, 0.0);
            for (int l = 0; l < P; ++l) {
                l2t[(size_t)(b * K + a) * P2 + 2 * l] = pw.real();
                l2t[(size_t)(b * K + a) * P2 + 2 * l + 1] = -pw.imag();
                pw *= xi;
            }
        }
    std::vector<double> C = binom_table(2 * P + 2);
    auto Cb = [&](int n, int k) { return (k < 0 || k > n) ? 0.0 : C[(size_t)n * (2 * P + 3) + k]; };
    // M2M / L2L: child position c, delta = child centre - parent centre in parent sides
    m2m.assign((size_t)4 * P2 * P2, 0.0);
    l2l.assign((size_t)4 * P2 * P2, 0.0);
    for (int c = 0; c < 4; ++c) {
        cd delta(((c & 1) - 0.5) * 0.5, ((c >> 1) - 0.5) * 0.5);
        std::vector<cd> dp(2 * P + 1);
        dp[0] = 1.0;
        for (int i = 1; i <= 2 * P; ++i) dp[i] = dp[i - 1] * delta;
        std::vector<cd> M((size_t)P * P, cd(0, 0)), LL((size_t)P * P, cd(0, 0));
        M[0] = 1.0;
        for (int l = 1; l < P; ++l) {
            M[(size_t)l * P] = -dp[l] / double(l);
            for (int k = 1; k <= l; ++k) M[(size_t)l * P + k] = dp[l - k] * (std::ldexp(1.0, -k) * Cb(l - 1, k - 1));
        }
        for (int m = 0; m < P; ++m)
            for (int l = m; l < P; ++l) LL[(size_t)m * P + l] = dp[l - m] * (std::ldexp(1.0, -m) * Cb(l, m));
        real_form(M, P, m2m, (size_t)c * P2 * P2);
        real_form(LL, P, l2l, (size_t)c * P2 * P2);
    }
    // M2L per list-i offset t (source - target, in box sides); a_0 log L is added separately
    m2l.assign((size_t)kVSlots * P2 * P2, 0.0);
    int idx = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            if (x >= -1 && x <= 1 && y >= -1 && y <= 1) continue;
            cd tt(x, y), it = 1.0 / tt;
            std::vector<cd> ip(2 * P + 1), mp(2 * P + 1);   // t^-n, (-t)^-n
            ip[0] = mp[0] = 1.0;
            for (int n = 1; n <= 2 * P; ++n) {
                ip[n] = ip[n - 1] * it;
                mp[n] = mp[n - 1] * (-it);
            }
            std::vector<cd> M((size_t)P * P, cd(0, 0));
            M[0] = std::log(std::abs(tt));   // Re log(-t)
            for (int k = 1; k < P; ++k) M[k] = mp[k];
            for (int l = 1; l < P; ++l) {
                M[(size_t)l * P] = -ip[l] / double(l);
                for (int k = 1; k < P; ++k) M[(size_t)l * P + k] = ip[l] * mp[k] * Cb(l + k - 1, k - 1);
            }
            real_form(M, P, m2l, (size_t)idx * P2 * P2);
            ++idx;
        }
    // M2T per list-i- position: zeta_i = (z_i - c_W) / L_W; row i: (log|zeta|, 0, Re zeta^-k, -Im zeta^-k)
    m2t.assign((size_t)kWSlots * KK * P2, 0.0);
    idx = 0;
    for (int y = -2; y <= 3; ++y)
        for (int x = -2; x <= 3; ++x) {
            if (x >= -1 && x <= 2 && y >= -1 && y <= 2) continue;
            for (int b = 0; b < K; ++b)
                for (int a = 0; a < K; ++a) {
                    cd zeta(1.0 + t[a] - (x + 0.5), 1.0 + t[b] - (y + 0.5));
                    double *row = &m2t[((size_t)idx * KK + b * K + a) * P2];
                    row[0] = std::log(std::abs(zeta));
                    cd iz = 1.0 / zeta, pw = 1.0;
                    for (int k = 1; k < P; ++k) {
                        pw *= iz;
                        row[2 * k] = pw.real();
                        row[2 * k + 1] = -pw.imag();
                    }
                }
            ++idx;
        }
}

// ------------------------------------------------------------- setup

void setup_chains(vpx_plan *p, const std::vector<double> &m2m, const std::vector<double> &l2l);   // chain.cu
void free_chains(vpx_plan *p);
void chain_reset(vpx_plan *p, cudaStream_t s);
void chain_run(vpx_plan *p, bool up, double *x, int64_t ldm, int nrhs, cudaStream_t s);


// The level chains as one persistent launch each in the FP64 form, one launch
// per level in the mixed form: measured on the L-shape step, the persistent
// chains cut the FP64 form's L2L from 0.38 to 0.14 ms, while the mixed form's
// double-float row engine per level ran as fast as they did beside the
// near-field kernel (0.684 against 0.692 ms per step).  VPX_PERSISTENT_CHAINS
// (1 or 0) overrides the choice for either form.
static bool use_chains(const vpx_plan *p) {
    if (!p->fmm.chain.ok) return false;
    const char *e = getenv("VPX_PERSISTENT_CHAINS");
    if (e) return e[0] == '1';
    return p->opt.precision != VPX_PREC_MIXED;
}

void setup_passes(vpx_plan *p) {
    const bool mixed = p->opt.precision == VPX_PREC_MIXED;
    const int KK = p->KK, P = p->P, P2 = 2 * P, nl = (int)p->tree.leaves.size(), nb = (int)p->box_level.size();
    std::vector<double> l2m, l2t, m2m, l2l, m2l, m2t;
    fmm_tables_host(p, l2m, l2t, m2m, l2l, m2l, m2t);
    std::vector<double> near((size_t)kNearConfigs * KK * KK);
    VPX_CUDA(cudaMemcpy(near.data(), p->tab.near, near.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> s2l_dev((size_t)kXSlots * KK * P * 2), s2l((size_t)kXSlots * P2 * KK);
    VPX_CUDA(cudaMemcpy(s2l_dev.data(), p->tab.s2l, s2l_dev.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int c = 0; c < kXSlots; ++c)   // device layout [c][j][l] complex -> [c][2P][KK]
        for (int j = 0; j < KK; ++j)
            for (int l = 0; l < P; ++l) {
                s2l[((size_t)c * P2 + 2 * l) * KK + j] = s2l_dev[(((size_t)c * KK + j) * P + l) * 2];
                s2l[((size_t)c * P2 + 2 * l + 1) * KK + j] = s2l_dev[(((size_t)c * KK + j) * P + l) * 2 + 1];
            }
    auto lvl_side = [](int l) { return std::ldexp(1.0, -l); };
    std::vector<int32_t> leaf_box(nl);
    for (int b = 0; b < nb; ++b)
        if (p->box_leaf[b] >= 0) leaf_box[p->box_leaf[b]] = b;
    FmmPasses &F = p->fmm;
    typedef std::vector<std::pair<int, GPair>> Tagged;
    // L2M
    {
        Tagged tg;
        for (int i = 0; i < nl; ++i)
            if (p->leaf_nz[i]) {
                double h = 0.5 * lvl_side(p->tree.leaves[i].level);
                tg.push_back({0, GPair{i, 0, (int64_t)leaf_box[i] * P2, h * h}});
            }
        gemm_pass_upload_tables(F.l2m, l2m, 1, P2, KK, mixed);
        F.l2m.add = 1;   // into the zeroed multipoles (the inner dimension may be split)
        gemm_pass_set_pairs(F.l2m, tg);
    }
    // The level chains in bands of levels, one launch per band.  In the scaled
    // variables a translation does not depend on the level, so the translation
    // across d levels is a product of d of the four child tables: 4^d tables of
    // depth d, from index (4^d - 4) / 3 on, numbered by the child positions
    // along the path, pos_1 (the lower box in its parent) + 4 pos_2 + ...
    //  Upward (M2M), bands of up to kBandUp levels: a launch reads every box
    //  at level L (final after the band below) and the leaves of the levels
    //  between L and the band's top level Lt = max(L - kBandUp, 2) (final from
    //  L2M), and adds each one's translation into each of its ancestors down to
    //  Lt.  It writes only boxes with children, at levels Lt .. L-1, and reads
    //  only boxes at L and leaves, so no box is read and written in one launch;
    //  every leaf's multipole reaches every ancestor once, through the boxes of
    //  the levels read.
    //  Downward (L2L), bands of two levels: lo(g) = lo'(g) + T lo'(c) + T T lo(a)
    //  for g below c below a, lo' a box's own terms (M2L, lists i+, constants).
    //  A first launch adds T lo'(c) for the boxes c of the levels between the
    //  read levels; then a launch per band reads the final lo(a) at level L and
    //  adds it into the children (depth 1) and grandchildren (depth 2).
    for (int l = 0; l <= kMaxLevel; ++l) {
        F.m2m[l] = GemmPass();
        F.l2l[l] = GemmPass();
    }
    F.n_m2m = F.n_l2l = 0;
    {
        constexpr int kBandUp = 3;
        const int D = p->n_levels - 1;
        const size_t T2 = (size_t)P2 * P2;
        auto off = [](int d) { return ((1 << (2 * d)) - 4) / 3; };
        // tables of depths 1 .. depth, composed in FP64: upward T[pos_d] ... T[pos_1],
        // downward T[pos_1] ... T[pos_d]
        auto band_tables = [&](const std::vector<double> &t4, int depth, bool up, int &ntab) {
            ntab = off(depth + 1);
            std::vector<double> all((size_t)ntab * T2, 0.0);
            std::copy(t4.begin(), t4.begin() + 4 * T2, all.begin());
            for (int d = 2; d <= depth; ++d)
                for (int code = 0; code < (1 << (2 * d)); ++code) {
                    const int cp = code & ((1 << (2 * (d - 1))) - 1), pd = code >> (2 * (d - 1));
                    const double *A = up ? &t4[pd * T2] : &all[(off(d - 1) + cp) * T2];
                    const double *B = up ? &all[(off(d - 1) + cp) * T2] : &t4[pd * T2];
                    double *C = &all[(off(d) + code) * T2];
                    for (int i = 0; i < P2; ++i)
                        for (int j = 0; j < P2; ++j) {
                            const double a = A[(size_t)i * P2 + j];
                            if (a == 0.0) continue;
                            for (int k = 0; k < P2; ++k) C[(size_t)i * P2 + k] += a * B[(size_t)j * P2 + k];
                        }
                }
            return all;
        };
        int ntu = 0, ntd = 0;
        const std::vector<double> tu = band_tables(m2m, kBandUp, true, ntu), td = band_tables(l2l, 2, false, ntd);
        gemm_pass_upload_tables(F.m2m_tab, tu, ntu, P2, P2, mixed);
        gemm_pass_upload_tables(F.l2l_tab, td, ntd, P2, P2, mixed);
        if (mixed) {   // the level chains: double-float row engine
            gemm_pass_use_rows(F.m2m_tab, tu);
            gemm_pass_use_rows(F.l2l_tab, td);
        }
        for (int L = D; L > 2;) {
            const int Lt = std::max(L - kBandUp, 2);
            Tagged tm;
            for (int b = p->level_start[Lt + 1]; b < p->level_start[L + 1]; ++b) {
                if (!p->box_nz[b] || (p->box_level[b] < L && p->box_child0[b] >= 0)) continue;
                int c = b, code = 0, d = 0;
                for (;;) {
                    const int a = p->box_parent[c];
                    if (a < 0 || p->box_level[a] < Lt) break;
                    code += (c - p->box_child0[a]) << (2 * d);
                    ++d;
                    tm.push_back({off(d) + code, GPair{b, 0, (int64_t)a * P2, 1.0}});
                    c = a;
                }
            }
            gemm_pass_view(F.m2m[F.n_m2m], F.m2m_tab);
            gemm_pass_set_pairs(F.m2m[F.n_m2m], tm);
            ++F.n_m2m;
            L = Lt;
        }
        Tagged pre;
        for (int L = 2; L + 1 <= D; L += 2) {
            Tagged tl;
            for (int a = p->level_start[L]; a < p->level_start[L + 1]; ++a) {
                const int c0 = p->box_child0[a];
                if (c0 < 0) continue;
                for (int i = 0; i < 4; ++i) {
                    const int c = c0 + i, g0 = p->box_child0[c];
                    tl.push_back({off(1) + i, GPair{a, 0, (int64_t)c * P2, 1.0}});
                    if (g0 < 0) continue;
                    for (int j = 0; j < 4; ++j) {
                        tl.push_back({off(2) + j + 4 * i, GPair{a, 0, (int64_t)(g0 + j) * P2, 1.0}});
                        pre.push_back({off(1) + j, GPair{c, 0, (int64_t)(g0 + j) * P2, 1.0}});
                    }
                }
            }
            gemm_pass_view(F.l2l[F.n_l2l], F.l2l_tab);
            gemm_pass_set_pairs(F.l2l[F.n_l2l], tl);
            ++F.n_l2l;
        }
        gemm_pass_view(F.l2l_pre, F.l2l_tab);
        gemm_pass_set_pairs(F.l2l_pre, pre);
    }
    // M2L and S2L
    {
        Tagged tv, tx;
        for (int b = p->level_start[std::min(2, p->n_levels)]; b < nb; ++b) {
            for (int s = 0; s < kVSlots; ++s) {
                int src = p->vlist[(size_t)b * kVSlots + s];
                if (src >= 0) tv.push_back({s, GPair{src, 0, (int64_t)b * P2, 1.0}});
            }
            for (int s = 0; s < kXSlots; ++s) {
                int src = p->xlist[(size_t)b * kXSlots + s];
                if (src >= 0) {
                    double H = 0.5 * lvl_side(p->tree.leaves[src].level);
                    tx.push_back({s, GPair{src, 0, (int64_t)b * P2, H * H}});
                }
            }
        }
        gemm_pass_upload_tables(F.m2l, m2l, kVSlots, P2, P2, mixed);
        gemm_pass_set_pairs(F.m2l, tv);
        gemm_pass_upload_tables(F.s2l, s2l, kXSlots, P2, KK, mixed);
        gemm_pass_set_pairs(F.s2l, tx, 32);   // third stream: fewer, fuller CTAs leave the main chain room
    }
    // L2T, M2T, near: the factor 1/2pi of the kernel is folded into the tables, so
    // that every pair scale of every pass is a power of two (h^2 or 1)
    {
        const double inv2pi = 0.15915494309189533576888376337251;
        for (std::vector<double> *t : {&l2t, &m2t, &near})
            for (double &x : *t) x *= inv2pi;
        Tagged tt, tw, tn;
        for (int i = 0; i < nl; ++i) {
            if (p->tree.leaves[i].level >= 2) tt.push_back({0, GPair{leaf_box[i], 0, (int64_t)i * KK, 1.0}});
            for (int s = 0; s < kWSlots; ++s) {
                int wb = p->wlist[(size_t)i * kWSlots + s];
                if (wb >= 0) tw.push_back({s, GPair{wb, 0, (int64_t)i * KK, 1.0}});
            }
            for (int c = 0; c < kNearConfigs; ++c) {
                int src = p->near[(size_t)i * kNearConfigs + c];
                if (src >= 0) {
                    double h = 0.5 * lvl_side(p->tree.leaves[src].level);
                    tn.push_back({c, GPair{src, 0, (int64_t)i * KK, h * h}});
                }
            }
        }
        gemm_pass_upload_tables(F.l2t, l2t, 1, KK, P2, mixed);
        gemm_pass_set_pairs(F.l2t, tt);
        gemm_pass_upload_tables(F.m2t, m2t, kWSlots, KK, P2, mixed);
        gemm_pass_set_pairs(F.m2t, tw, 32);
        gemm_pass_upload_tables(F.near, near, kNearConfigs, KK, KK, mixed);
        gemm_pass_set_pairs(F.near, tn);
    }
    // gather lists of the level-dependent constant terms
    {
        const double ln2 = std::log(2.0), inv2pi = 0.15915494309189533576888376337251;
        std::vector<int32_t> off(1, 0), idx;
        std::vector<double> coef;
        F.lc_first = p->level_start[std::min(2, p->n_levels)];
        for (int b = F.lc_first; b < nb; ++b) {
            for (int s2 = 0; s2 < kVSlots; ++s2) {
                const int src = p->vlist[(size_t)b * kVSlots + s2];
                if (src >= 0) {
                    idx.push_back(src);
                    coef.push_back(-(double)p->box_level[b] * ln2);
                }
            }
            for (int s2 = 0; s2 < kXSlots; ++s2) {
                const int src = p->xlist[(size_t)b * kXSlots + s2];
                if (src >= 0) {
                    idx.push_back(leaf_box[src]);
                    coef.push_back(-(double)(p->tree.leaves[src].level + 1) * ln2);
                }
            }
            off.push_back((int32_t)idx.size());
        }
        F.lc_rows = nb - F.lc_first;
        F.lc_off = dev_upload(off);
        F.lc_idx = dev_upload(idx);
        F.lc_coef = dev_upload(coef);
        off.assign(1, 0);
        idx.clear();
        coef.clear();
        for (int i = 0; i < nl; ++i) {
            for (int c = 0; c < kNearConfigs; ++c) {
                const int src = p->near[(size_t)i * kNearConfigs + c];
                if (src >= 0) {
                    idx.push_back(leaf_box[src]);
                    coef.push_back(-(double)(p->tree.leaves[src].level + 1) * ln2 * inv2pi);
                }
            }
            for (int s2 = 0; s2 < kWSlots; ++s2) {
                const int wb = p->wlist[(size_t)i * kWSlots + s2];
                if (wb >= 0) {
                    idx.push_back(wb);
                    coef.push_back(-(double)p->box_level[wb] * ln2 * inv2pi);
                }
            }
            off.push_back((int32_t)idx.size());
        }
        F.tc_off = dev_upload(off);
        F.tc_idx = dev_upload(idx);
        F.tc_coef = dev_upload(coef);
    }
    if (mixed) {
        gemm_ws_prepare_device();
        gemm_frag_prepare_device();
        for (GemmPass *g : {&F.near, &F.l2m, &F.m2l, &F.s2l, &F.l2t, &F.m2t}) gemm_ws_prepare(*g);
        // M2L starts on the mma.sync engine: its 2(p+1)-row tables fill under
        // half of a 128-row tcgen05 block and its inner dimension is one or two
        // stages deep, so a tcgen05 tile is mostly set-up (measured on the
        // L-shape at p = 27: 0.147 ms on tcgen05 against 0.090 ms).  The
        // autotuner keeps tcgen05 as a candidate.
        F.m2l.engine = 1;
        const int kp_f = (KK + 31) / 32 * 32, kp_m = (P2 + 31) / 32 * 32;
        F.fe_sl = dev_alloc<uint16_t>((size_t)p->opt.max_rhs * nl * kSlicesS * kp_f);
        F.fe_ex = dev_alloc<int32_t>((size_t)p->opt.max_rhs * nl);
        F.mp_sl = dev_alloc<uint16_t>((size_t)p->opt.max_rhs * nb * kSlicesS * kp_m);
        F.mp_ex = dev_alloc<int32_t>((size_t)p->opt.max_rhs * nb);
    }
    for (GemmPass *g : {&F.l2m, &F.m2l, &F.s2l, &F.l2t, &F.m2t, &F.near}) g->status = p->wk.status;
    for (int l = 0; l <= kMaxLevel; ++l) F.m2m[l].status = F.l2l[l].status = p->wk.status;
    for (GemmPass *g : {&F.m2m_tab, &F.l2l_tab, &F.l2l_pre}) g->status = p->wk.status;
    setup_chains(p, m2m, l2l);
    VPX_CUDA(cudaDeviceSynchronize());
}

void free_passes(vpx_plan *p) {
    FmmPasses &F = p->fmm;
    free_chains(p);
    gemm_pass_free(F.l2m);
    gemm_pass_free(F.m2l);
    gemm_pass_free(F.s2l);
    gemm_pass_free(F.l2t);
    gemm_pass_free(F.m2t);
    gemm_pass_free(F.near);
    for (int l = 0; l <= kMaxLevel; ++l) {
        gemm_pass_free(F.m2m[l]);
        gemm_pass_free(F.l2l[l]);
    }
    gemm_pass_free(F.l2l_pre);
    gemm_pass_free(F.m2m_tab);
    gemm_pass_free(F.l2l_tab);
    dev_free(F.fe_sl);
    dev_free(F.fe_ex);
    dev_free(F.lc_off);
    dev_free(F.lc_idx);
    dev_free(F.lc_coef);
    dev_free(F.tc_off);
    dev_free(F.tc_idx);
    dev_free(F.tc_coef);
    dev_free(F.mp_sl);
    dev_free(F.mp_ex);
}

// ------------------------------------------------------------ execute

void ev_record_pass(vpx_plan *p, int i, cudaStream_t s);

// Three streams forked from the main one: the near field (leaf values only)
// on the second; list i+ (leaf values -> locals) and, once the multipoles are
// final, the a_0 log terms of the locals and of V and list i- on the third.
// They overlap the level-by-level passes of the main stream, add into V or the
// locals with atomics, and are joined where their results are read (the
// locals before L2L, V before the last launch).
void run_potential_passes(vpx_plan *p, const double *fe, int64_t ldfe, int nrhs, double *v, int64_t ldv, double *vb,
                          int64_t ldb, double *mp, double *lo, cudaStream_t s, bool fe_sliced) {
    const bool mixed = p->opt.precision == VPX_PREC_MIXED;
    const int P = p->P, P2 = 2 * P, KK = p->KK;
    const DevTree &d = p->dt;
    const int nb = d.n_boxes, nl = d.n_leaves;
    const int64_t ldm = (int64_t)nb * P2;
    const int kp_f = (KK + 31) / 32 * 32, kp_m = (P2 + 31) / 32 * 32;
    FmmPasses &F = p->fmm;
    VecSet vf{fe, ldfe, KK, F.fe_sl, F.fe_ex, nl, kp_f};
    // expansions along the level chains are sliced by the pass that reads them;
    // the final multipoles once, for lists i and i-
    VecSet vm{mp, ldm, P2, nullptr, nullptr, nb, 0};
    VecSet vl{lo, ldm, P2, nullptr, nullptr, nb, 0};
    VecSet vmf{mp, ldm, P2, F.mp_sl, F.mp_ex, nb, kp_m};
    if (!mixed) vmf = vm;
    cudaStream_t aux = (cudaStream_t)p->aux_stream, aux2 = (cudaStream_t)p->aux2_stream;
    LaunchPriority critical(priority_greatest());
    ev_record_pass(p, 1, s);
    VPX_CUDA(cudaMemsetAsync(mp, 0, sizeof(double) * ldm * nrhs, s));
    VPX_CUDA(cudaMemsetAsync(lo, 0, sizeof(double) * ldm * nrhs, s));
    const bool chains = use_chains(p);
    if (chains) chain_reset(p, s);
    VPX_CUDA(cudaMemset2DAsync(v, sizeof(double) * ldv, 0, sizeof(double) * (size_t)nl * KK, nrhs, s));
    // the leaf-value slices serve L2M, the near field and list i+ (slicing L2M's
    // 256-long vectors on the fly took longer than slicing once before it)
    if (mixed && !fe_sliced) slice_vectors(vf, 0, nl, KK, kp_f, nrhs, s);
    // fork: the near field on the second stream; list i+ (leaf values ->
    // local), then the constant terms and list i- on the third
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_fork, s));
    VPX_CUDA(cudaStreamWaitEvent(aux, (cudaEvent_t)p->ev_fork, 0));
    VPX_CUDA(cudaStreamWaitEvent(aux2, (cudaEvent_t)p->ev_fork, 0));
    ev_record_pass(p, VPX_N_PASSES + 1, aux);
    {
        LaunchPriority background(priority_least());
        gemm_run(F.near, vf, v, ldv, nrhs, mixed, aux);
    }
    ev_record_pass(p, VPX_N_PASSES + 2, aux);
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_join, aux));
    gemm_run(F.s2l, vf, lo, ldm, nrhs, mixed, aux2);
    // main stream: upward pass
    gemm_run(F.l2m, vf, mp, ldm, nrhs, mixed, s);
    ev_record_pass(p, 2, s);
    if (chains) chain_run(p, true, mp, ldm, nrhs, s);
    else
        for (int k = 0; k < F.n_m2m; ++k) gemm_run(F.m2m[k], vm, mp, ldm, nrhs, mixed, s);
    if (mixed) slice_vectors(vmf, 0, nb, P2, kp_m, nrhs, s);
    // the final multipoles feed the constant terms and list i- on the third
    // stream, beside M2L on this one (all accumulate into distinct sums)
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_up, s));
    VPX_CUDA(cudaStreamWaitEvent(aux2, (cudaEvent_t)p->ev_up, 0));
    if (F.lc_rows > 0) {
        launch_pdl(k_const_gather, dim3((F.lc_rows + 7) / 8, nrhs), dim3(256), 0, aux2, 
            F.lc_rows, F.lc_first, P, F.lc_off, F.lc_idx, F.lc_coef, mp, ldm, lo, ldm, P2, 1);
        VPX_LAUNCH("k_const_gather");
    }
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_lc, aux2));   // list i+ and local constants done
    gemm_run(F.m2t, vmf, v, ldv, nrhs, mixed, aux2);
    if (nl > 0) {
        launch_pdl(k_const_gather, dim3((nl + 7) / 8, nrhs), dim3(256), 0, aux2, nl, 0, P, F.tc_off, F.tc_idx, F.tc_coef, mp, ldm,
                                                                   v, ldv, KK, KK);
        VPX_LAUNCH("k_const_gather");
    }
    VPX_CUDA(cudaEventRecord((cudaEvent_t)p->ev_join2, aux2));
    ev_record_pass(p, 3, s);
    gemm_run(F.m2l, vmf, lo, ldm, nrhs, mixed, s);
    VPX_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)p->ev_lc, 0));
    ev_record_pass(p, 4, s);
    if (chains) {
        chain_run(p, false, lo, ldm, nrhs, s);
    } else {
        gemm_run(F.l2l_pre, vl, lo, ldm, nrhs, mixed, s);
        for (int k = 0; k < F.n_l2l; ++k) gemm_run(F.l2l[k], vl, lo, ldm, nrhs, mixed, s);
    }
    ev_record_pass(p, 5, s);
    gemm_run(F.l2t, vl, v, ldv, nrhs, mixed, s);
    ev_record_pass(p, 6, s);
    VPX_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)p->ev_join, 0));
    VPX_CUDA(cudaStreamWaitEvent(s, (cudaEvent_t)p->ev_join2, 0));
    ev_record_pass(p, 7, s);
}

}  // namespace vpx
