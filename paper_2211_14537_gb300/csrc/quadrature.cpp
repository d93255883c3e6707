// quadrature.cpp -- point sets and quadrature rules used by the library's setup.
//
// Gauss-Legendre nodes (leaf grids, boundary panels; Sections 4 and 5),
// Chebyshev nodes of the first kind (extension square, Section 3.2),
// Padua points (our choice of the Gaussian support set G, Section 3.2), and a
// Gauss rule for the weight -r log r on [0,1] used to integrate the log kernel
// in polar coordinates when the near-field tables are generated.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace vpx {

uint32_t morton2(uint32_t ix, uint32_t iy) {
    uint32_t k = 0;
    for (int b = 0; b < 16; ++b) {
        k |= ((ix >> b) & 1u) << (2 * b);
        k |= ((iy >> b) & 1u) << (2 * b + 1);
    }
    return k;
}

// Legendre P_n and P_n' by the three-term recurrence.
static void legendre_pd(int n, double x, double &p, double &dp) {
    double a = 1.0, b = x;
    if (n == 0) {
        p = 1.0;
        dp = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    p = b;
    dp = n * (a - x * b) / (1.0 - x * x);
}

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 0; k < (n + 1) / 2; ++k) {
        // Tricomi's asymptotic guess for the k-th root counted from x = 1
        double th = kPi * (4.0 * k + 3.0) / (4.0 * n + 2.0);
        double r = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
        double p = 0, dp = 1;
        for (int it = 0; it < 60; ++it) {
            legendre_pd(n, r, p, dp);
            double step = p / dp;
            r -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        legendre_pd(n, r, p, dp);
        x[n - 1 - k] = r;
        x[k] = -r;
        double wk = 2.0 / ((1.0 - r * r) * dp * dp);
        w[n - 1 - k] = wk;
        w[k] = wk;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

// Gauss rule for the weight w(r) = -r log(r) on [0, 1], n nodes:
// recurrence coefficients by the discretised Stieltjes procedure (the
// measure discretised by Gauss-Legendre panels graded toward r = 0), nodes as
// roots of the n-th orthogonal polynomial, weights as Christoffel numbers.
void gauss_log_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    std::vector<double> g, gw;
    gauss_legendre(30, g, gw);
    std::vector<double> rr, ww;
    double hi = 1.0;
    for (int panel = 0; panel < 80; ++panel) {
        double lo = hi * 0.5;
        if (panel == 79) lo = 0.0;
        for (size_t i = 0; i < g.size(); ++i) {
            double r = 0.5 * (lo + hi) + 0.5 * (hi - lo) * g[i];
            rr.push_back(r);
            ww.push_back(0.5 * (hi - lo) * gw[i] * (-r * std::log(r)));
        }
        hi = lo;
    }
    const size_t M = rr.size();
    std::vector<double> alpha(n), beta(n);
    std::vector<double> pm1(M, 0.0), p0(M, 1.0), p1(M);
    double nrm_prev = 0.0;
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0, s = 0.0;
        for (size_t i = 0; i < M; ++i) {
            nrm += ww[i] * p0[i] * p0[i];
            s += ww[i] * rr[i] * p0[i] * p0[i];
        }
        alpha[k] = s / nrm;
        beta[k] = (k == 0) ? nrm : nrm / nrm_prev;
        nrm_prev = nrm;
        for (size_t i = 0; i < M; ++i) {
            p1[i] = (rr[i] - alpha[k]) * p0[i] - (k == 0 ? 0.0 : beta[k]) * pm1[i];
        }
        pm1.swap(p0);
        p0.swap(p1);
    }
    // monic recurrence evaluation of pi_n (value) at r
    auto eval = [&](double r, std::vector<double> *vals) {
        double a = 0.0, b = 1.0;
        if (vals) (*vals)[0] = 1.0;
        for (int k = 0; k < n; ++k) {
            double c = (r - alpha[k]) * b - (k == 0 ? 0.0 : beta[k]) * a;
            a = b;
            b = c;
            if (vals && k + 1 < n) (*vals)[k + 1] = b;
        }
        return b;
    };
    // roots: scan for sign changes on a fine grid, then bisection
    x.clear();
    const int NS = 20000;
    double prev_r = 0.0, prev_v = eval(0.0, nullptr);
    for (int i = 1; i <= NS; ++i) {
        double r = double(i) / NS;
        r = r * r;  // denser near 0
        double v = eval(r, nullptr);
        if ((v > 0) != (prev_v > 0)) {
            double lo = prev_r, hi2 = r, vlo = prev_v;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi2);
                double vm = eval(mid, nullptr);
                if ((vm > 0) == (vlo > 0)) {
                    lo = mid;
                    vlo = vm;
                } else {
                    hi2 = mid;
                }
                if (hi2 - lo < 1e-17) break;
            }
            x.push_back(0.5 * (lo + hi2));
        }
        prev_r = r;
        prev_v = v;
    }
    if ((int)x.size() != n) fail(VPX_ERR_ARG, "gauss_log_rule: root count mismatch");
    // Christoffel numbers with the orthonormal polynomials
    w.assign(n, 0.0);
    std::vector<double> vals(n);
    for (int i = 0; i < n; ++i) {
        eval(x[i], &vals);
        double s = 0.0, nk = beta[0];
        for (int k = 0; k < n; ++k) {
            if (k > 0) nk *= beta[k];
            s += vals[k] * vals[k] / nk;
        }
        w[i] = 1.0 / s;
    }
}

std::vector<double> chebyshev1(int n) {
    std::vector<double> t(n);
    for (int a = 0; a < n; ++a) t[a] = -std::cos((2.0 * a + 1.0) * kPi / (2.0 * n));
    return t;
}

void padua(int q, std::vector<double> &x, std::vector<double> &y) {
    x.clear();
    y.clear();
    for (int j = 0; j <= q; ++j)
        for (int k = 0; k <= q + 1; ++k)
            if ((j + k) % 2 == 0) {
                x.push_back(std::cos(j * kPi / q));
                y.push_back(std::cos(k * kPi / (q + 1)));
            }
}

std::vector<double> barycentric_weights(const std::vector<double> &t) {
    std::vector<double> bw(t.size());
    for (size_t a = 0; a < t.size(); ++a) {
        double p = 1.0;
        for (size_t m = 0; m < t.size(); ++m)
            if (m != a) p *= (t[a] - t[m]);
        bw[a] = 1.0 / p;
    }
    return bw;
}

// Lagrange basis values at s by the barycentric formula (exact node hits handled).
void lagrange_eval(const std::vector<double> &t, const std::vector<double> &bw, double s, double *out) {
    const size_t K = t.size();
    for (size_t a = 0; a < K; ++a)
        if (s == t[a]) {
            for (size_t m = 0; m < K; ++m) out[m] = (m == a) ? 1.0 : 0.0;
            return;
        }
    double den = 0.0;
    for (size_t a = 0; a < K; ++a) {
        out[a] = bw[a] / (s - t[a]);
        den += out[a];
    }
    for (size_t a = 0; a < K; ++a) out[a] /= den;
}

}  // namespace vpx
