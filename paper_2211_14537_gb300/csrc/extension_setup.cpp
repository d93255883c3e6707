// extension_setup.cpp -- universal stencil and per-cut-leaf extension operators.
//
// Section 3.2: for a cut leaf S with extension square Sbar (side 3L, same
// centre), the universal point set is X_S (the K x K leaf nodes), X_Sbar (a
// Kbar x Kbar Chebyshev grid of the first kind on Sbar) and the support set G.
// The universal matrix A_{X,G} = Phi_{X,G} Phi_{G,G}^{-1} maps values at G to
// values at X; for each cut leaf the rows of the interior points give A_I and
// the extension is f_{X_Sbar^E} = A_{X_Sbar^E,G} A_I^+ f_I.
//
// By default the Gaussian basis is read in its flat limit (shape parameter ->
// 0): with G unisolvent for the polynomials P_q of total degree <= q and
// N_G = dim P_q, A is the Lagrange interpolation matrix of P_q at G.  With a
// positive shape parameter the eps^2 term of the Gaussian operator is added
// from a table precomputed in multiprecision (universal_operator).  G is
// the Padua point set of degree q = 10 (N_G = 66, Section 6), Kbar = 3K/2.  A is formed with the
// well-conditioned tensor Chebyshev basis T_m T_n (m + n <= q), and A_I^+ (the
// Moore-Penrose pseudo-inverse) by Householder QR plus a one-sided Jacobi SVD
// of the triangular factor; singular values below 1e-13 of the largest are
// dropped, which also covers cut leaves with fewer than N_G interior points.  The apply on the device stores P_S = A_I^+ per cut
// leaf (N_G x N_I, row-major) and the universal rows A_{X_Sbar,G}.
#include <algorithm>
#include <cmath>
#include <thread>

#include "internal.h"

namespace vpx {

namespace {

// T_0..T_q at x
void cheb_values(int q, double x, double *out) {
    out[0] = 1.0;
    if (q >= 1) out[1] = x;
    for (int m = 2; m <= q; ++m) out[m] = 2.0 * x * out[m - 1] - out[m - 2];
}

// Phi row: T_m(x) T_n(y), m + n <= q, ordered by m then n
void phi_row(int q, double x, double y, double *row) {
    double tx[64], ty[64];
    cheb_values(q, x, tx);
    cheb_values(q, y, ty);
    int c = 0;
    for (int m = 0; m <= q; ++m)
        for (int n = 0; n + m <= q; ++n) row[c++] = tx[m] * ty[n];
}

// Solve M X = B (M n x n row-major, B n x r row-major) by LU with partial pivoting.
void lu_solve(int n, std::vector<double> M, std::vector<double> &B, int r) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(M[i * n + k]) > std::fabs(M[p * n + k])) p = i;
        if (M[p * n + k] == 0.0) fail(VPX_ERR_STENCIL, "singular interpolation matrix at G");
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(M[k * n + j], M[p * n + j]);
            for (int j = 0; j < r; ++j) std::swap(B[k * r + j], B[p * r + j]);
        }
        for (int i = k + 1; i < n; ++i) {
            double f = M[i * n + k] / M[k * n + k];
            if (f == 0.0) continue;
            for (int j = k; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
            for (int j = 0; j < r; ++j) B[i * r + j] -= f * B[k * r + j];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        for (int j = 0; j < r; ++j) {
            double s = B[k * r + j];
            for (int i = k + 1; i < n; ++i) s -= M[k * n + i] * B[i * r + j];
            B[k * r + j] = s / M[k * n + k];
        }
    }
}

constexpr double kPinvRcond = 1e-13;   // singular values below this fraction of the largest are dropped

// Householder QR of a (rows x cols, rows >= cols, column-major): returns the
// thin Q (rows x cols, column-major) and R (cols x cols, row-major).
void householder_qr(int rows, int cols, std::vector<double> &a, std::vector<double> &Q, std::vector<double> &R) {
    std::vector<double> V((size_t)rows * cols, 0.0);
    R.assign((size_t)cols * cols, 0.0);
    for (int k = 0; k < cols; ++k) {
        double *x = &a[(size_t)k * rows];
        double nrm = 0.0;
        for (int i = k; i < rows; ++i) nrm += x[i] * x[i];
        nrm = std::sqrt(nrm);
        double alpha = (x[k] > 0) ? -nrm : nrm;
        double *v = &V[(size_t)k * rows];
        for (int i = k; i < rows; ++i) v[i] = x[i];
        v[k] -= alpha;
        double vn = 0.0;
        for (int i = k; i < rows; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        if (vn > 0)
            for (int i = k; i < rows; ++i) v[i] /= vn;
        for (int j = k; j < cols; ++j) {
            double *c = &a[(size_t)j * rows];
            double s = 0.0;
            for (int i = k; i < rows; ++i) s += v[i] * c[i];
            for (int i = k; i < rows; ++i) c[i] -= 2.0 * s * v[i];
        }
        for (int j = k; j < cols; ++j) R[(size_t)k * cols + j] = a[(size_t)j * rows + k];
    }
    Q.assign((size_t)rows * cols, 0.0);
    for (int j = 0; j < cols; ++j) Q[(size_t)j * rows + j] = 1.0;
    for (int k = cols - 1; k >= 0; --k) {
        const double *v = &V[(size_t)k * rows];
        for (int j = 0; j < cols; ++j) {
            double *c = &Q[(size_t)j * rows];
            double s = 0.0;
            for (int i = k; i < rows; ++i) s += v[i] * c[i];
            for (int i = k; i < rows; ++i) c[i] -= 2.0 * s * v[i];
        }
    }
}

// One-sided (Hestenes) Jacobi SVD of the n x n matrix R (row-major):
// R W = U Sigma with W orthogonal.  On return U holds the columns R W
// (column-major, unnormalised), W the right singular vectors (column-major),
// sig the column norms.
void jacobi_svd(int n, const std::vector<double> &R, std::vector<double> &U, std::vector<double> &W,
                std::vector<double> &sig) {
    U.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) U[(size_t)j * n + i] = R[(size_t)i * n + j];
    W.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) W[(size_t)j * n + j] = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double *up = &U[(size_t)p * n], *uq = &U[(size_t)q * n];
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < n; ++i) {
                    al += up[i] * up[i];
                    be += uq[i] * uq[i];
                    ga += up[i] * uq[i];
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-16 * std::sqrt(al * be)) continue;
                off = std::max(off, std::fabs(ga) / std::sqrt(al * be));
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < n; ++i) {
                    double a = up[i], b = uq[i];
                    up[i] = c * a - s * b;
                    uq[i] = s * a + c * b;
                }
                double *wp = &W[(size_t)p * n], *wq = &W[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    double a = wp[i], b = wq[i];
                    wp[i] = c * a - s * b;
                    wq[i] = s * a + c * b;
                }
            }
        if (off < 1e-15) break;
    }
    sig.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += U[(size_t)j * n + i] * U[(size_t)j * n + i];
        sig[j] = std::sqrt(s);
    }
}

// P = A_I^+ (n x m, row-major) for A_I (m x n, row-major): Moore-Penrose
// pseudo-inverse, singular values <= kPinvRcond * sigma_max treated as zero.
// QR of A_I (or of A_I^T when m < n) reduces it to a square triangular
// factor whose SVD is taken by one-sided Jacobi.  Returns the condition
// number of the kept part and the infinity norm of P.
void pseudo_inverse(int m, int n, const double *AI, double *P, double *cond, double *pnorm) {
    const bool tall = m >= n;
    const int rows = tall ? m : n, cols = tall ? n : m;
    std::vector<double> a((size_t)rows * cols);   // column-major rows x cols
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            if (tall) a[(size_t)j * m + i] = AI[(size_t)i * n + j];
            else a[(size_t)i * n + j] = AI[(size_t)i * n + j];   // A^T column i = row i of A
        }
    std::vector<double> Q, R, U, W, sig;
    householder_qr(rows, cols, a, Q, R);
    jacobi_svd(cols, R, U, W, sig);
    double smax = 0.0;
    for (double s : sig) smax = std::max(smax, s);
    double smin_kept = smax;
    // Z = W Sigma^+ Uhat^T  (cols x cols), Uhat = U / sigma
    std::vector<double> Z((size_t)cols * cols, 0.0);
    for (int k = 0; k < cols; ++k) {
        if (!(sig[k] > kPinvRcond * smax)) continue;
        smin_kept = std::min(smin_kept, sig[k]);
        double inv2 = 1.0 / (sig[k] * sig[k]);
        const double *wk = &W[(size_t)k * cols], *uk = &U[(size_t)k * cols];
        for (int i = 0; i < cols; ++i)
            for (int j = 0; j < cols; ++j) Z[(size_t)i * cols + j] += wk[i] * uk[j] * inv2;
    }
    // tall:  R = Uhat S W^T, A = Q R  =>  A^+ = W S^+ Uhat^T Q^T = Z Q^T
    // wide:  A^T = Q R, A = R^T Q^T, R^T = W S Uhat^T  =>  A^+ = Q Uhat S^+ W^T = Q Z^T
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            if (tall)
                for (int k = 0; k < cols; ++k) s += Z[(size_t)i * cols + k] * Q[(size_t)k * rows + j];
            else
                for (int k = 0; k < cols; ++k) s += Q[(size_t)k * rows + i] * Z[(size_t)j * cols + k];
            P[(size_t)i * m + j] = s;
        }
    double pn = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += std::fabs(P[(size_t)i * m + j]);
        pn = std::max(pn, s);
    }
    *pnorm = pn;
    *cond = smax / smin_kept;
}

}  // namespace

// Stencil of the extension along lines (Section 6.4): per cut leaf its interior
// leaf nodes X_S^I and grid points X_Sbar^I, then for each exterior grid point
// (grid order) the kRayNodes points at radii r_b - j L / kRayNodes, j = 1..,
// on the line from the origin through it, where r_b is the boundary radius in
// that direction and L the leaf side.  r_b is found by bisection on the inside
// test between the origin (inside: Omega is star-shaped about it) and the grid
// point (outside), all lines at once, one callback per step.
constexpr int kRayNodes = 8;

// Floater-Hormann weights of degree d on the nodes x[0..n] (any order):
// w_k = (-1)^(k-d) sum_{i in J_k} prod_{j=i..i+d, j != k} 1/|x_k - x_j| with the
// nodes sorted ascending; the coefficients of the interpolant at z follow as
// (w_k / (z - x_k)) / sum_i w_i / (z - x_i), returned in the order of x.
static void fh_coefficients(const double *x, int n1, int d, double z, double *coef) {
    std::vector<int> ord(n1);
    for (int k = 0; k < n1; ++k) ord[k] = k;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return x[a] < x[b]; });
    const int n = n1 - 1;
    std::vector<double> xs(n1), w(n1);
    for (int k = 0; k < n1; ++k) xs[k] = x[ord[k]];
    for (int k = 0; k <= n; ++k) {
        double tot = 0.0;
        for (int i = std::max(0, k - d); i <= std::min(k, n - d); ++i) {
            double p = 1.0;
            for (int j = i; j <= i + d; ++j)
                if (j != k) p /= std::fabs(xs[k] - xs[j]);
            tot += p;
        }
        w[k] = ((k - d) % 2 == 0 ? 1.0 : -1.0) * tot;
    }
    double den = 0.0;
    for (int k = 0; k <= n; ++k) den += w[k] / (z - xs[k]);
    for (int k = 0; k <= n; ++k) coef[ord[k]] = w[k] / (z - xs[k]) / den;
}

constexpr int kRayDegree = 3;   // Floater-Hormann blending degree (the text leaves it open)

void ray_stencil(const vpx_options &opt, const Callbacks &cb, const HostTree &tree, StencilInfo &st,
                 const std::vector<double> &cxy, const std::vector<uint8_t> &ins, int NX, int KK, int KbKb,
                 std::vector<double> &stencil_xy) {
    const int ncut = (int)st.cut_leaf.size();
    std::vector<double> ux, uy, rp, lside;
    std::vector<int> owner_c, grid_e;
    for (int c = 0; c < ncut; ++c) {
        const double L = std::ldexp(1.0, -tree.leaves[st.cut_leaf[c]].level);
        for (int e = 0; e < KbKb; ++e) {
            const size_t j = (size_t)c * NX + KK + e;
            if (ins[j]) continue;
            const double x = cxy[2 * j], y = cxy[2 * j + 1], r = std::hypot(x, y);
            if (!(r > 0.0)) fail(VPX_ERR_STENCIL, "a grid point at the origin");
            ux.push_back(x / r);
            uy.push_back(y / r);
            rp.push_back(r);
            lside.push_back(L);
            owner_c.push_back(c);
            grid_e.push_back(e);
        }
    }
    const size_t nr = rp.size();
    std::vector<double> lo(nr, 0.0), hi = rp, pts(2 * nr);
    std::vector<uint8_t> in(nr);
    for (int it = 0; it < 64 && nr; ++it) {
        for (size_t k = 0; k < nr; ++k) {
            const double m = 0.5 * (lo[k] + hi[k]);
            pts[2 * k] = m * ux[k];
            pts[2 * k + 1] = m * uy[k];
        }
        if (cb.inside(pts.data(), (int64_t)nr, in.data(), cb.ctx) != 0) fail(VPX_ERR_CALLBACK, "inside callback failed");
        for (size_t k = 0; k < nr; ++k) {
            const double m = 0.5 * (lo[k] + hi[k]);
            (in[k] ? lo[k] : hi[k]) = m;
        }
    }
    st.mode = 1;
    st.stencil_off.assign(ncut, 0);
    st.n_interior.assign(ncut, 0);
    st.grid_src.assign((size_t)ncut * KbKb, -1);
    st.node_src.assign((size_t)ncut * KK, -1);
    st.ray_c.clear();
    st.ray_g.clear();
    st.ray_src.clear();
    st.ray_coef.clear();
    size_t k = 0;
    double rad[kRayNodes], coef[kRayNodes];
    for (int c = 0; c < ncut; ++c) {
        st.stencil_off[c] = (int64_t)(stencil_xy.size() / 2);
        int cnt = 0;
        for (int j = 0; j < KK + KbKb; ++j) {
            if (!ins[(size_t)c * NX + j]) continue;
            if (j < KK) st.node_src[(size_t)c * KK + j] = cnt;
            else st.grid_src[(size_t)c * KbKb + (j - KK)] = cnt;
            stencil_xy.push_back(cxy[2 * ((size_t)c * NX + j)]);
            stencil_xy.push_back(cxy[2 * ((size_t)c * NX + j) + 1]);
            ++cnt;
        }
        for (; k < nr && owner_c[k] == c; ++k) {
            st.ray_c.push_back(c);
            st.ray_g.push_back(grid_e[k]);
            st.ray_src.push_back(st.stencil_off[c] + cnt);
            for (int q = 1; q <= kRayNodes; ++q) {
                rad[q - 1] = lo[k] - lside[k] * q / kRayNodes;
                if (!(rad[q - 1] > 0.0)) fail(VPX_ERR_STENCIL, "ray points reach the origin");
                stencil_xy.push_back(rad[q - 1] * ux[k]);
                stencil_xy.push_back(rad[q - 1] * uy[k]);
            }
            fh_coefficients(rad, kRayNodes, kRayDegree, rp[k], coef);
            for (int q = 0; q < kRayNodes; ++q) st.ray_coef.push_back(coef[q]);
            cnt += kRayNodes;
        }
        st.n_interior[c] = cnt;
    }
    // The construction assumes a domain star-shaped about the origin: every
    // ray point lies between the origin and the ray's one boundary crossing.
    // Refuse a geometry where that fails (the exterior of inclusions, say)
    // rather than extend from points outside Omega.
    std::vector<double> rxy;
    for (size_t r = 0; r < st.ray_src.size(); ++r)
        for (int q = 0; q < kRayNodes; ++q) {
            const size_t p = (size_t)st.ray_src[r] + q;
            rxy.push_back(stencil_xy[2 * p]);
            rxy.push_back(stencil_xy[2 * p + 1]);
        }
    const size_t nrp = rxy.size() / 2;
    std::vector<uint8_t> rin(nrp);
    if (nrp && cb.inside(rxy.data(), (int64_t)nrp, rin.data(), cb.ctx) != 0)
        fail(VPX_ERR_CALLBACK, "inside callback failed");
    for (size_t p = 0; p < nrp; ++p)
        if (!rin[p]) fail(VPX_ERR_STENCIL, "extension along lines: a ray point lies outside Omega "
                                           "(the domain is not star-shaped about the origin)");
    (void)opt;
}

void check_rbf_eps(int K, double rbf_eps) {
    if (!(rbf_eps >= 0.0) || rbf_eps > 1e-3) fail(VPX_ERR_ARG, "rbf_eps must lie in [0, 1e-3]");
    const double *a2 = nullptr;
    int nx = 0, ng = 0;
    if (rbf_eps > 0.0 && !rbf_eps2_table(K, &a2, &nx, &ng))
        fail(VPX_ERR_ARG, "rbf_eps > 0 needs K = 6, 8 or 16 (no Gaussian table for this K)");
}

// A = Phi_X Phi_G^{-1} in the flat limit (the Lagrange basis of P_q at G,
// formed with the tensor Chebyshev basis), plus (rbf_eps / 2)^2 A2 for
// Gaussians of shape parameter rbf_eps on the unit box: the extension square
// maps to [-1,1]^2, whose side is twice the unit box's, and the remainder of
// the series is O(rbf_eps^4), below 1e-13 for rbf_eps <= 1e-3.
void universal_operator(int K, double rbf_eps, std::vector<double> &A, int &NX, int &NG) {
    const int q = 10, Kb = 3 * K / 2, KK = K * K, KbKb = Kb * Kb;
    NG = (q + 1) * (q + 2) / 2;
    NX = KK + KbKb + NG;
    std::vector<double> t, tw;
    gauss_legendre(K, t, tw);
    std::vector<double> tc = chebyshev1(Kb);
    std::vector<double> px, py;
    padua(q, px, py);
    if ((int)px.size() != NG) fail(VPX_ERR_ARG, "Padua point count mismatch");
    std::vector<double> xy(2 * (size_t)NX);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a) {
            xy[2 * (b * K + a)] = t[a] / 3.0;
            xy[2 * (b * K + a) + 1] = t[b] / 3.0;
        }
    for (int b = 0; b < Kb; ++b)
        for (int a = 0; a < Kb; ++a) {
            xy[2 * (KK + b * Kb + a)] = tc[a];
            xy[2 * (KK + b * Kb + a) + 1] = tc[b];
        }
    for (int g = 0; g < NG; ++g) {
        xy[2 * (KK + KbKb + g)] = px[g];
        xy[2 * (KK + KbKb + g) + 1] = py[g];
    }
    // solve Phi_G^T Y = Phi_X^T, A = Y^T
    std::vector<double> PhiG((size_t)NG * NG), B((size_t)NG * NX), row(NG);
    for (int g = 0; g < NG; ++g) {
        phi_row(q, px[g], py[g], row.data());
        for (int k = 0; k < NG; ++k) PhiG[(size_t)k * NG + g] = row[k];   // transpose
    }
    for (int j = 0; j < NX; ++j) {
        phi_row(q, xy[2 * j], xy[2 * j + 1], row.data());
        for (int k = 0; k < NG; ++k) B[(size_t)k * NX + j] = row[k];
    }
    lu_solve(NG, PhiG, B, NX);
    A.assign((size_t)NX * NG, 0.0);
    for (int j = 0; j < NX; ++j)
        for (int k = 0; k < NG; ++k) A[(size_t)j * NG + k] = B[(size_t)k * NX + j];
    if (rbf_eps > 0.0) {
        const double *a2 = nullptr;
        int nx = 0, ng = 0;
        if (!rbf_eps2_table(K, &a2, &nx, &ng) || nx != NX || ng != NG)
            fail(VPX_ERR_ARG, "no Gaussian table matching this universal stencil");
        const double e = 0.5 * rbf_eps, e2 = e * e;
        for (size_t i = 0; i < A.size(); ++i) A[i] += e2 * a2[i];
    }
}

void build_stencil(const vpx_options &opt, const Callbacks &cb, const HostTree &tree,
                   std::vector<double> &stencil_xy, StencilInfo &st, bool compute_operators) {
    const int K = opt.K, KK = K * K;
    st.q = 10;   // N_G = 66 support points (Section 6) for every K
    st.Kbar = 3 * K / 2;
    st.NG = (st.q + 1) * (st.q + 2) / 2;
    const int Kb = st.Kbar, KbKb = Kb * Kb, NG = st.NG;
    st.NX = KK + KbKb + NG;
    const int NX = st.NX;

    std::vector<double> t, tw;
    gauss_legendre(K, t, tw);
    std::vector<double> tc = chebyshev1(Kb);
    std::vector<double> px, py;
    padua(st.q, px, py);
    if ((int)px.size() != NG) fail(VPX_ERR_ARG, "Padua point count mismatch");

    st.ref_xy.assign(2 * (size_t)NX, 0.0);
    for (int b = 0; b < K; ++b)
        for (int a = 0; a < K; ++a) {
            st.ref_xy[2 * (b * K + a)] = t[a] / 3.0;
            st.ref_xy[2 * (b * K + a) + 1] = t[b] / 3.0;
        }
    for (int b = 0; b < Kb; ++b)
        for (int a = 0; a < Kb; ++a) {
            st.ref_xy[2 * (KK + b * Kb + a)] = tc[a];
            st.ref_xy[2 * (KK + b * Kb + a) + 1] = tc[b];
        }
    for (int g = 0; g < NG; ++g) {
        st.ref_xy[2 * (KK + KbKb + g)] = px[g];
        st.ref_xy[2 * (KK + KbKb + g) + 1] = py[g];
    }

    // stencil points: regular leaves, then the interior stencil of each cut leaf
    const int nl = (int)tree.leaves.size();
    st.reg_leaf_off.assign(nl, -1);
    stencil_xy.clear();
    for (int i = 0; i < nl; ++i) {
        const Leaf &L = tree.leaves[i];
        if (L.cls != kRegular) continue;
        st.reg_leaf_off[i] = (int64_t)(stencil_xy.size() / 2);
        double s = std::ldexp(1.0, -L.level), h = 0.5 * s;
        double cx = -0.5 + (L.ix + 0.5) * s, cy = -0.5 + (L.iy + 0.5) * s;
        for (int b = 0; b < K; ++b)
            for (int a = 0; a < K; ++a) {
                stencil_xy.push_back(cx + h * t[a]);
                stencil_xy.push_back(cy + h * t[b]);
            }
    }
    st.cut_leaf.clear();
    for (int i = 0; i < nl; ++i)
        if (tree.leaves[i].cls == kCut) st.cut_leaf.push_back(i);
    const int ncut = (int)st.cut_leaf.size();
    // physical stencil points of all cut leaves, one batched inside() call
    std::vector<double> cxy((size_t)ncut * NX * 2);
    for (int c = 0; c < ncut; ++c) {
        const Leaf &L = tree.leaves[st.cut_leaf[c]];
        double s = std::ldexp(1.0, -L.level);
        double cx = -0.5 + (L.ix + 0.5) * s, cy = -0.5 + (L.iy + 0.5) * s;
        for (int j = 0; j < NX; ++j) {
            double zx = st.ref_xy[2 * j], zy = st.ref_xy[2 * j + 1];
            if (j < KK) {   // leaf nodes exactly as the regular leaves compute them
                cxy[2 * ((size_t)c * NX + j)] = cx + 0.5 * s * t[j % K];
                cxy[2 * ((size_t)c * NX + j) + 1] = cy + 0.5 * s * t[j / K];
            } else {
                cxy[2 * ((size_t)c * NX + j)] = cx + 1.5 * s * zx;
                cxy[2 * ((size_t)c * NX + j) + 1] = cy + 1.5 * s * zy;
            }
        }
    }
    std::vector<uint8_t> ins((size_t)ncut * NX, 0);
    if (ncut && cb.inside(cxy.data(), (int64_t)ins.size(), ins.data(), cb.ctx) != 0)
        fail(VPX_ERR_CALLBACK, "inside callback failed");
    std::vector<std::vector<int>> interior(ncut);
    if (opt.ext_mode == 1) {   // extension along lines (Section 6.4): no support set G in the stencil
        ray_stencil(opt, cb, tree, st, cxy, ins, NX, KK, KbKb, stencil_xy);
    } else {
    st.mode = 0;
    st.stencil_off.assign(ncut, 0);
    st.n_interior.assign(ncut, 0);
    st.grid_src.assign((size_t)ncut * KbKb, -1);
    st.node_src.assign((size_t)ncut * KK, -1);
    for (int c = 0; c < ncut; ++c) {
        st.stencil_off[c] = (int64_t)(stencil_xy.size() / 2);
        int cnt = 0;
        for (int j = 0; j < NX; ++j) {
            if (!ins[(size_t)c * NX + j]) continue;
            if (j < KK) st.node_src[(size_t)c * KK + j] = cnt;
            else if (j < KK + KbKb) st.grid_src[(size_t)c * KbKb + (j - KK)] = cnt;
            interior[c].push_back(j);
            stencil_xy.push_back(cxy[2 * ((size_t)c * NX + j)]);
            stencil_xy.push_back(cxy[2 * ((size_t)c * NX + j) + 1]);
            ++cnt;
        }
        st.n_interior[c] = cnt;
    }
    }
    // owned exterior leaves per cut leaf
    std::vector<int> cut_index(nl, -1);
    for (int c = 0; c < ncut; ++c) cut_index[st.cut_leaf[c]] = c;
    std::vector<std::vector<int>> owned(ncut);
    for (int i = 0; i < nl; ++i)
        if (tree.leaves[i].owner >= 0) owned[cut_index[tree.leaves[i].owner]].push_back(i);
    st.owned_off.assign(ncut + 1, 0);
    st.owned.clear();
    for (int c = 0; c < ncut; ++c) {
        st.owned_off[c + 1] = st.owned_off[c] + (int)owned[c].size();
        for (int i : owned[c]) st.owned.push_back(i);
    }
    // Chebyshev transform on the Kbar grid: alpha_m = sum_a C[m][a] F_a
    st.cheb_inv.assign((size_t)KbKb, 0.0);
    {
        double tv[64];
        for (int a = 0; a < Kb; ++a) {
            cheb_values(Kb - 1, tc[a], tv);
            for (int m = 0; m < Kb; ++m) st.cheb_inv[m * Kb + a] = (m == 0 ? 1.0 : 2.0) / Kb * tv[m];
        }
    }
    if (!compute_operators || st.mode == 1) return;   // mode 1: the line coefficients are the operator

    // the universal A (flat limit, plus the Gaussian eps^2 term when rbf_eps > 0)
    {
        int nx = 0, ng = 0;
        universal_operator(K, opt.rbf_eps, st.A, nx, ng);
        if (nx != NX || ng != NG) fail(VPX_ERR_ARG, "universal stencil size mismatch");
    }

    st.pinv_off.assign(ncut, 0);
    size_t tot = 0;
    for (int c = 0; c < ncut; ++c) {
        if (st.n_interior[c] < 1) fail(VPX_ERR_STENCIL, "cut leaf without interior stencil points");
        st.pinv_off[c] = (int64_t)tot;
        tot += (size_t)NG * st.n_interior[c];
    }
    st.pinv.assign(tot, 0.0);
    std::vector<double> norms(ncut, 0.0), conds(ncut, 0.0);
    unsigned nth = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    auto work = [&](unsigned tid) {
        std::vector<double> AI;
        for (int c = (int)tid; c < ncut; c += (int)nth) {
            int m = st.n_interior[c];
            AI.assign((size_t)m * NG, 0.0);
            for (int r = 0; r < m; ++r) {
                int j = interior[c][r];
                std::copy(&st.A[(size_t)j * NG], &st.A[(size_t)j * NG] + NG, &AI[(size_t)r * NG]);
            }
            pseudo_inverse(m, NG, AI.data(), &st.pinv[st.pinv_off[c]], &conds[c], &norms[c]);
        }
    };
    std::vector<std::thread> th;
    for (unsigned i = 0; i < nth; ++i) th.emplace_back(work, i);
    for (auto &x : th) x.join();
    for (int c = 0; c < ncut; ++c) {
        st.max_pinv_norm = std::max(st.max_pinv_norm, norms[c]);
        st.max_cond = std::max(st.max_cond, conds[c]);
    }
}

}  // namespace vpx
