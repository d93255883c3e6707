// bie_setup.cpp -- host part of the boundary correction (Section 5); for the
// interior Dirichlet problem on a simply connected domain
//
//   u = V[f^e] + D[sigma],  (-1/2 + D)[sigma] = g - V[f^e] on Gamma,
//   D[sigma](x) = int (1/2pi) (x - y).nu(y) / |x - y|^2 sigma(y) ds_y,
//
// nu the outward normal (eqs. dlpot, dblker, inteq).  The Nystrom
// discretisation uses the panels' Gauss-Legendre nodes with s = |gamma'| and
// the weights w (eq. discdblpotpanel); on the diagonal the kernel takes its
// limit on the boundary, -kappa / (4 pi).  Near a panel the Gauss-Legendre sum
// loses accuracy; there the panel's contribution is integrated exactly
// against the polynomial through its nodes (Helsing-Ojala product
// integration, named in Section 5): in complex form a panel contributes
// -(1/2pi) Im int sigma(tau) dtau / (tau - z).  This file computes the
// geometry and, for every leaf node within reach of a panel, the weights that
// replace that panel's plain terms.  With several closed curves (holes, or the
// inclusions of an exterior problem, Section 2) each curve is classified by
// the side Omega lies on, which sets the jump of its double layer: -1/2 on
// Omega's outer boundary, +1/2 on a curve Omega surrounds (every curve
// counter-clockwise, nu pointing out of the region it encloses).
#include <algorithm>
#include <cmath>
#include <complex>
#include <thread>

#include "internal.h"
#include "plan.h"

namespace vpx {

using cplx = std::complex<double>;

namespace {

constexpr double kNearRadius = 2.0;   // product integration when |zeta| < 2 (panel coordinates)

// Differentiation matrix at the nodes t (barycentric form): Dm[j][k] =
// (bw_k / bw_j) / (t_j - t_k), diagonal minus the row sum.
std::vector<double> diff_matrix(const std::vector<double> &t, const std::vector<double> &bw) {
    const int n = (int)t.size();
    std::vector<double> Dm((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double diag = 0.0;
        for (int k = 0; k < n; ++k)
            if (k != j) {
                Dm[(size_t)j * n + k] = (bw[k] / bw[j]) / (t[j] - t[k]);
                diag -= Dm[(size_t)j * n + k];
            }
        Dm[(size_t)j * n + j] = diag;
    }
    return Dm;
}

// Value of the interpolant through (t_j, v_j) at s (barycentric, second form).
cplx interp(const std::vector<double> &t, const std::vector<double> &bw, const cplx *v, double s) {
    cplx num = 0.0;
    double den = 0.0;
    for (size_t j = 0; j < t.size(); ++j) {
        const double d = s - t[j];
        if (d == 0.0) return v[j];
        num += v[j] * (bw[j] / d);
        den += bw[j] / d;
    }
    return num / den;
}

// Solve the complex n x n system M x = r in place (partial pivoting); M row-major.
void csolve(int n, std::vector<cplx> &M, std::vector<cplx> &r) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int i = c + 1; i < n; ++i)
            if (std::abs(M[(size_t)i * n + c]) > std::abs(M[(size_t)piv * n + c])) piv = i;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(M[(size_t)c * n + k], M[(size_t)piv * n + k]);
            std::swap(r[c], r[piv]);
        }
        const cplx d = M[(size_t)c * n + c];
        for (int i = c + 1; i < n; ++i) {
            const cplx f = M[(size_t)i * n + c] / d;
            if (f == cplx(0.0)) continue;
            for (int k = c; k < n; ++k) M[(size_t)i * n + k] -= f * M[(size_t)c * n + k];
            r[i] -= f * r[c];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        cplx s = r[i];
        for (int k = i + 1; k < n; ++k) s -= M[(size_t)i * n + k] * r[k];
        r[i] = s / M[(size_t)i * n + i];
    }
}

struct PanelData {
    std::vector<double> t, bw, Dm;
};

// lam with sum_j lam_j sigma_j = int_panel sigma dtau / (tau - z), sigma the
// polynomial of degree nq - 1 in xi = (2 tau - a - b) / (b - a) through the
// nodes: lam solves V^T lam = p with V[j][k] = xi_j^k and p_k = int xi^k /
// (xi - zeta) dxi along the panel (p_k = zeta p_{k-1} + (1 - (-1)^k) / k).
void product_weights(const PanelData &P, const cplx *tau, cplx a, cplx b, cplx z, cplx *lam) {
    const int n = (int)P.t.size();
    std::vector<cplx> xi(n), dxi(n, 0.0);
    for (int j = 0; j < n; ++j) xi[j] = (2.0 * tau[j] - (a + b)) / (b - a);
    const cplx zeta = (2.0 * z - (a + b)) / (b - a);
    std::vector<cplx> p(n);
    p[0] = std::log((1.0 - zeta) / (-1.0 - zeta));     // along the chord [-1, 1]
    if (std::fabs(zeta.real()) < 1.0) {
        // height of the curved panel where its real part is Re(zeta): Newton on
        // the interpolant xi(t), derivative from the differentiation matrix
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) dxi[j] += P.Dm[(size_t)j * n + k] * xi[k];
        double s = zeta.real();
        for (int it = 0; it < 60; ++it) {
            const double f = interp(P.t, P.bw, xi.data(), s).real() - zeta.real();
            const double step = f / interp(P.t, P.bw, dxi.data(), s).real();
            s -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        const double h = interp(P.t, P.bw, xi.data(), s).imag();
        // between the panel and its chord the two integrals differ by the residue
        if (h != 0.0 && zeta.imag() / h > 0.0 && zeta.imag() / h < 1.0)
            p[0] += cplx(0.0, h > 0.0 ? -2.0 * M_PI : 2.0 * M_PI);
    }
    for (int k = 1; k < n; ++k) p[k] = zeta * p[k - 1] + ((k % 2) ? 2.0 / k : 0.0);
    std::vector<cplx> VT((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        cplx pw = 1.0;
        for (int k = 0; k < n; ++k) {
            VT[(size_t)k * n + j] = pw;
            pw *= xi[j];
        }
    }
    csolve(n, VT, p);
    for (int j = 0; j < n; ++j) lam[j] = p[j];
}

// Closed curves: a curve runs over consecutive panels, each starting where the
// previous one ends, until one ends where the curve's first panel starts.
// Returns the first panel of every curve, then the panel count.
std::vector<int> split_curves(const vpx_plan *pl) {
    const int np = (int)(pl->bdry_ends.size() / 4);
    const double *E = pl->bdry_ends.data();
    double len = 0.0;
    for (int i = 0; i < np; ++i) len += std::hypot(E[4 * i + 2] - E[4 * i], E[4 * i + 3] - E[4 * i + 1]);
    const double tol = 1e-10 * len;
    auto meets = [&](int i, int k) { return std::hypot(E[4 * i + 2] - E[4 * k], E[4 * i + 3] - E[4 * k + 1]) <= tol; };
    std::vector<int> first_panel;
    for (int i = 0; i < np;) {
        const int f = i;
        while (i < np && !meets(i, f)) {
            if (i + 1 >= np || !meets(i, i + 1))
                fail(VPX_ERR_STATE, "the boundary correction needs closed curves (panel ends must meet)");
            ++i;
        }
        first_panel.push_back(f);
        ++i;
    }
    first_panel.push_back(np);
    return first_panel;
}

// Normals, s*w, curvature and the curve of every node; every curve must be
// counter-clockwise (positive signed area, twice it = int (x y' - y x') dt).
void node_geometry(const vpx_plan *pl, const std::vector<int> &first, const PanelData &P, const std::vector<double> &w,
                   BieHost &B) {
    const int nq = B.nq, nc = B.n_curves;
    const size_t N = pl->bdry_xy.size() / 2;
    B.nu.assign(2 * N, 0.0);
    B.sw.assign(N, 0.0);
    B.kappa.assign(N, 0.0);
    B.curve_of_node.assign(N, 0);
    std::vector<double> area2(nc, 0.0);
    for (int c = 0; c < nc; ++c)
        for (int i = first[c]; i < first[c + 1]; ++i)
            for (int j = 0; j < nq; ++j) {
                const size_t q = (size_t)i * nq + j;
                const double dx = pl->bdry_dxy[2 * q], dy = pl->bdry_dxy[2 * q + 1];
                double ddx = 0.0, ddy = 0.0;
                for (int k = 0; k < nq; ++k) {
                    ddx += P.Dm[(size_t)j * nq + k] * pl->bdry_dxy[2 * ((size_t)i * nq + k)];
                    ddy += P.Dm[(size_t)j * nq + k] * pl->bdry_dxy[2 * ((size_t)i * nq + k) + 1];
                }
                const double s = std::hypot(dx, dy);
                B.nu[2 * q] = dy / s;
                B.nu[2 * q + 1] = -dx / s;
                B.sw[q] = s * w[j];
                B.kappa[q] = (dx * ddy - dy * ddx) / (s * s * s);
                B.curve_of_node[q] = c;
                area2[c] += w[j] * (pl->bdry_xy[2 * q] * dy - pl->bdry_xy[2 * q + 1] * dx);
            }
    for (int c = 0; c < nc; ++c)
        if (!(area2[c] > 0.0)) fail(VPX_ERR_STATE, "the boundary correction needs counter-clockwise curves");
}

// The side of Omega: a point just off the middle node of each curve's first
// panel, along the curve's outward normal, is in Omega exactly when Omega lies
// outside the curve (a hole, or an inclusion of an exterior problem: jump
// +1/2); otherwise the curve is Omega's outer boundary (-1/2).
void curve_sides(const vpx_plan *pl, const std::vector<int> &first, BieHost &B, vpx_inside_cb inside, void *ctx) {
    const int nq = B.nq, nc = B.n_curves;
    const double *E = pl->bdry_ends.data();
    std::vector<double> probe(2 * nc);
    for (int c = 0; c < nc; ++c) {
        const size_t q = (size_t)first[c] * nq + nq / 2;
        const int f = first[c];
        const double L = std::hypot(E[4 * f + 2] - E[4 * f], E[4 * f + 3] - E[4 * f + 1]);
        probe[2 * c] = pl->bdry_xy[2 * q] + 1e-3 * L * B.nu[2 * q];
        probe[2 * c + 1] = pl->bdry_xy[2 * q + 1] + 1e-3 * L * B.nu[2 * q + 1];
    }
    std::vector<uint8_t> in(nc);
    if (inside(probe.data(), nc, in.data(), ctx) != 0) fail(VPX_ERR_CALLBACK, "inside callback failed");
    B.outer_curve = -1;
    B.jump.assign(pl->bdry_xy.size() / 2, 0.0);
    for (int c = 0; c < nc; ++c) {
        if (!in[c]) {
            if (B.outer_curve >= 0) fail(VPX_ERR_STATE, "the boundary correction found two outer curves");
            B.outer_curve = c;
        }
        for (int i = first[c]; i < first[c + 1]; ++i)
            for (int j = 0; j < nq; ++j) B.jump[(size_t)i * nq + j] = in[c] ? 0.5 : -0.5;
    }
}

// One log term per curve that Omega surrounds, centred at the curve's area
// centroid (Green: A = 1/2 int (x y' - y x'), A cx = 1/2 int x^2 y',
// A cy = -1/2 int y^2 x'), which must lie outside Omega.
void log_terms(const vpx_plan *pl, const std::vector<int> &first, const std::vector<double> &w, BieHost &B,
               vpx_inside_cb inside, void *ctx) {
    const int nq = B.nq;
    B.log_curve.clear();
    B.log_centre.clear();
    for (int c = 0; c < B.n_curves; ++c) {
        if (c == B.outer_curve) continue;
        double a2 = 0.0, mx = 0.0, my = 0.0;
        for (int i = first[c]; i < first[c + 1]; ++i)
            for (int j = 0; j < nq; ++j) {
                const size_t q = (size_t)i * nq + j;
                const double x = pl->bdry_xy[2 * q], yq = pl->bdry_xy[2 * q + 1];
                const double dx = pl->bdry_dxy[2 * q], dy = pl->bdry_dxy[2 * q + 1];
                a2 += w[j] * (x * dy - yq * dx);
                mx += w[j] * x * x * dy;
                my -= w[j] * yq * yq * dx;
            }
        B.log_curve.push_back(c);
        B.log_centre.push_back(mx / a2);
        B.log_centre.push_back(my / a2);
    }
    B.n_log = (int)B.log_curve.size();
    if (B.n_log) {
        std::vector<uint8_t> cin(B.n_log);
        if (inside(B.log_centre.data(), B.n_log, cin.data(), ctx) != 0) fail(VPX_ERR_CALLBACK, "inside callback failed");
        for (int k = 0; k < B.n_log; ++k)
            if (cin[k]) fail(VPX_ERR_STATE, "the centroid of a hole or inclusion lies in Omega (no log centre)");
    }
    B.n_unknowns = (int)(pl->bdry_xy.size() / 2) + B.n_log;
}

// Product-integration corrections: for every (leaf node, panel) pair with
// |zeta| < kNearRadius, i.e. the node within |b - a| of the panel's chord
// midpoint (candidate leaves by box overlap), the Helsing-Ojala weights minus
// the panel's plain terms, CSR over the leaf nodes; computed on all cores.
void near_corrections(const vpx_plan *pl, const PanelData &P, BieHost &B) {
    const int nq = B.nq, np = B.n_panels;
    const double *E = pl->bdry_ends.data();
    const auto &L = pl->tree.leaves;
    const int KK = pl->KK;
    const size_t nt = pl->leaf_xy.size() / 2, N = pl->bdry_xy.size() / 2;
    std::vector<std::vector<int32_t>> near_of(nt);
    for (int i = 0; i < np; ++i) {
        const double mx = 0.5 * (E[4 * i] + E[4 * i + 2]), my = 0.5 * (E[4 * i + 1] + E[4 * i + 3]);
        const double R = kNearRadius * 0.5 * std::hypot(E[4 * i + 2] - E[4 * i], E[4 * i + 3] - E[4 * i + 1]);
        for (size_t l = 0; l < L.size(); ++l) {
            const double s = std::ldexp(1.0, -L[l].level);
            const double x0 = -0.5 + L[l].ix * s, y0 = -0.5 + L[l].iy * s;
            if (mx + R < x0 || mx - R > x0 + s || my + R < y0 || my - R > y0 + s) continue;
            for (int k = 0; k < KK; ++k) {
                const size_t q = l * KK + k;
                if (std::hypot(pl->leaf_xy[2 * q] - mx, pl->leaf_xy[2 * q + 1] - my) < R) near_of[q].push_back(i);
            }
        }
    }
    B.corr_off.assign(nt + 1, 0);
    for (size_t q = 0; q < nt; ++q) B.corr_off[q + 1] = B.corr_off[q] + (int64_t)near_of[q].size();
    const int64_t n_corr = B.corr_off[nt];
    B.corr_panel.assign(n_corr, 0);
    B.corr_w.assign((size_t)n_corr * nq, 0.0);
    for (size_t q = 0; q < nt; ++q)
        std::copy(near_of[q].begin(), near_of[q].end(), B.corr_panel.begin() + B.corr_off[q]);
    std::vector<cplx> tau(N);
    for (size_t q = 0; q < N; ++q) tau[q] = cplx(pl->bdry_xy[2 * q], pl->bdry_xy[2 * q + 1]);
    auto work = [&](size_t q0, size_t q1) {
        std::vector<cplx> lam(nq);
        for (size_t q = q0; q < q1; ++q) {
            const double x = pl->leaf_xy[2 * q], y = pl->leaf_xy[2 * q + 1];
            for (int64_t e = B.corr_off[q]; e < B.corr_off[q + 1]; ++e) {
                const int i = B.corr_panel[e];
                const cplx a(E[4 * i], E[4 * i + 1]), b(E[4 * i + 2], E[4 * i + 3]);
                product_weights(P, &tau[(size_t)i * nq], a, b, cplx(x, y), lam.data());
                for (int j = 0; j < nq; ++j) {
                    const size_t n = (size_t)i * nq + j;
                    const double dx = x - pl->bdry_xy[2 * n], dy = y - pl->bdry_xy[2 * n + 1];
                    const double plain = (dx * B.nu[2 * n] + dy * B.nu[2 * n + 1]) / (dx * dx + dy * dy) * B.sw[n];
                    B.corr_w[(size_t)e * nq + j] = (-lam[j].imag() - plain) / (2.0 * M_PI);
                }
            }
        }
    };
    const unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    const size_t chunk = (nt + nth - 1) / nth;
    for (unsigned k = 0; k < nth; ++k) {
        const size_t q0 = k * chunk, q1 = std::min(nt, q0 + chunk);
        if (q0 < q1) th.emplace_back(work, q0, q1);
    }
    for (auto &x : th) x.join();
}

// Each boundary node's double-layer term as a multipole of the leaf that holds
// it, in the box FMM's scaled form Phi(z) = a_0 log(z - c) + sum_k at_k
// (L / (z - c))^k, with (1/2pi) Re Phi the potential.  In complex form the node
// contributes Re(q / (z - tau)) with q = -i gamma'(t_j) w_j sigma / (2pi), and
// 1/(z - tau) = sum_{k>=1} (tau - c)^(k-1) / (z - c)^k, so for sigma = 1
//   a_0 = 0,  at_k = -i gamma' w (1/L) ((tau - c) / L)^(k-1).
void dipole_multipoles(const vpx_plan *pl, const std::vector<double> &w, BieHost &B) {
    const int nq = B.nq, P = pl->P;
    const size_t N = pl->bdry_xy.size() / 2;
    B.p2m.assign(N * 2 * P, 0.0);
    for (size_t q = 0; q < N; ++q) {
        const Leaf &lf = pl->tree.leaves[pl->bdry_leaf[q]];
        const double L = std::ldexp(1.0, -lf.level);
        const cplx c(-0.5 + (lf.ix + 0.5) * L, -0.5 + (lf.iy + 0.5) * L);
        const cplx tau(pl->bdry_xy[2 * q], pl->bdry_xy[2 * q + 1]);
        const cplx dtau(pl->bdry_dxy[2 * q], pl->bdry_dxy[2 * q + 1]);
        cplx a = cplx(0.0, -1.0) * dtau * (w[q % nq] / L);
        const cplx r = (tau - c) / L;
        for (int k = 1; k < P; ++k) {
            B.p2m[q * 2 * P + 2 * k] = a.real();
            B.p2m[q * 2 * P + 2 * k + 1] = a.imag();
            a *= r;
        }
    }
}

}  // namespace

void bie_setup(vpx_plan *pl, vpx_inside_cb inside, void *ctx) {
    BieHost &B = pl->bie;
    if (B.ready) return;
    if (pl->bdry_ends.empty()) fail(VPX_ERR_STATE, "the boundary correction needs boundary panels");
    const std::vector<int> first = split_curves(pl);
    B.nq = pl->opt.n_quad_bdry;
    B.n_panels = (int)(pl->bdry_ends.size() / 4);
    B.n_curves = (int)first.size() - 1;
    std::vector<double> t, w;
    gauss_legendre(B.nq, t, w);
    PanelData P{t, barycentric_weights(t), {}};
    P.Dm = diff_matrix(P.t, P.bw);
    node_geometry(pl, first, P, w, B);
    curve_sides(pl, first, B, inside, ctx);
    log_terms(pl, first, w, B, inside, ctx);
    near_corrections(pl, P, B);
    dipole_multipoles(pl, w, B);
    if (!pl->host_only) device_bie_setup(pl);
    B.ready = true;
}

}  // namespace vpx
