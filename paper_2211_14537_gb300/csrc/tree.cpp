// tree.cpp -- adaptive, level-restricted quad-tree on D = [-0.5,0.5]^2 (Section 4).
//
// Phase A (level by level): a box below min_level is split; otherwise, when
// adaptive, a box that is not exterior is split if f is not resolved on its
// K x K Gauss-Legendre grid (largest Legendre coefficient of total degree
// >= K-1 above refine_tol * f_scale; Section 4, adaptive refinement), and a
// cut box is split if its side exceeds twice the length of the shortest panel
// with a boundary sample inside it (Section 4, cut-size rule).
// Phase B (to a fixed point): 2:1 balance (level restriction), then the
// extension restriction: no exterior leaf coarser than a cut leaf S may
// overlap the extension square Sbar (Section 4).
// Classification: a leaf is cut when its K*K nodes straddle the boundary
// (some inside, some outside), regular when all are inside, exterior when
// all are outside.  Extension lists: an exterior leaf overlapping the
// extension squares of some cut leaves belongs to the one with the nearest
// centre; ties go to the cut leaf later in Z-order (Section 4).
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <unordered_set>

#include "internal.h"

namespace vpx {

namespace {

constexpr int kBoundarySamples = 64;   // intervals per panel for the cut-size rule

struct Geometry {
    std::vector<double> sx, sy;    // boundary samples
    std::vector<int32_t> spanel;   // panel of each sample
    std::vector<double> plen;      // panel lengths
};

void box_bounds(uint64_t k, double &x0, double &x1, double &y0, double &y1) {
    int l = key_level(k);
    double s = std::ldexp(1.0, -l);
    x0 = -0.5 + key_ix(k) * s;
    y0 = -0.5 + key_iy(k) * s;
    x1 = x0 + s;
    y1 = y0 + s;
}

uint64_t child_key(uint64_t k, int c) {
    return box_key(key_level(k) + 1, 2 * key_ix(k) + (c & 1), 2 * key_iy(k) + (c >> 1));
}

uint64_t ancestor_key(uint64_t k, int lev) {
    int sh = key_level(k) - lev;
    return box_key(lev, key_ix(k) >> sh, key_iy(k) >> sh);
}

struct Builder {
    const vpx_options &opt;
    const Callbacks &cb;
    std::vector<double> t, tw;           // leaf GL nodes / weights
    std::vector<double> Pm;              // Pm[m*K + a] = P_m(t_a)
    Geometry geo;
    std::unordered_map<uint64_t, int32_t> cls;

    Builder(const vpx_options &o, const Callbacks &c) : opt(o), cb(c) {
        gauss_legendre(opt.K, t, tw);
        Pm.assign(opt.K * opt.K, 0.0);
        for (int a = 0; a < opt.K; ++a) {
            double p0 = 1.0, p1 = t[a];
            Pm[a] = 1.0;
            if (opt.K > 1) Pm[opt.K + a] = t[a];
            for (int m = 2; m < opt.K; ++m) {
                double p2 = ((2 * m - 1) * t[a] * p1 - (m - 1) * p0) / m;
                p0 = p1;
                p1 = p2;
                Pm[m * opt.K + a] = p2;
            }
        }
        build_geometry();
    }

    void build_geometry() {
        std::vector<double> g, gw;
        gauss_legendre(16, g, gw);
        std::vector<double> ts(kBoundarySamples + 1);
        for (int m = 0; m <= kBoundarySamples; ++m) ts[m] = -1.0 + 2.0 * m / kBoundarySamples;
        std::vector<double> xy(2 * (kBoundarySamples + 1)), dxy(2 * (kBoundarySamples + 1));
        std::vector<double> xg(32), dg(32);
        for (int i = 0; i < cb.n_panels; ++i) {
            if (cb.curve(i, ts.data(), kBoundarySamples + 1, xy.data(), dxy.data(), cb.ctx) != 0)
                fail(VPX_ERR_CALLBACK, "curve callback failed");
            for (int m = 0; m <= kBoundarySamples; ++m) {
                geo.sx.push_back(xy[2 * m]);
                geo.sy.push_back(xy[2 * m + 1]);
                geo.spanel.push_back(i);
            }
            if (cb.curve(i, g.data(), 16, xg.data(), dg.data(), cb.ctx) != 0)
                fail(VPX_ERR_CALLBACK, "curve callback failed");
            double L = 0.0;
            for (int m = 0; m < 16; ++m) L += gw[m] * std::hypot(dg[2 * m], dg[2 * m + 1]);
            geo.plen.push_back(L);
        }
    }

    void nodes_of(uint64_t k, double *xy) const {
        double x0, x1, y0, y1;
        box_bounds(k, x0, x1, y0, y1);
        double cx = 0.5 * (x0 + x1), cy = 0.5 * (y0 + y1), h = 0.5 * (x1 - x0);
        const int K = opt.K;
        for (int b = 0; b < K; ++b)
            for (int a = 0; a < K; ++a) {
                xy[2 * (b * K + a)] = cx + h * t[a];
                xy[2 * (b * K + a) + 1] = cy + h * t[b];
            }
    }

    // classify every box of `ks` not yet classified (one batched callback)
    void classify(const std::vector<uint64_t> &ks) {
        std::vector<uint64_t> todo;
        for (uint64_t k : ks)
            if (!cls.count(k)) todo.push_back(k);
        if (todo.empty()) return;
        const int KK = opt.K * opt.K;
        std::vector<double> xy(2 * (size_t)KK * todo.size());
        for (size_t i = 0; i < todo.size(); ++i) nodes_of(todo[i], xy.data() + 2 * KK * i);
        std::vector<uint8_t> ins((size_t)KK * todo.size());
        if (cb.inside(xy.data(), (int64_t)ins.size(), ins.data(), cb.ctx) != 0)
            fail(VPX_ERR_CALLBACK, "inside callback failed");
        for (size_t i = 0; i < todo.size(); ++i) {
            int nin = 0;
            for (int j = 0; j < KK; ++j) nin += ins[KK * i + j] ? 1 : 0;
            cls[todo[i]] = (nin == KK) ? kRegular : (nin == 0 ? kExterior : kCut);
        }
    }

    double min_panel_len_in(uint64_t k) const {
        double x0, x1, y0, y1;
        box_bounds(k, x0, x1, y0, y1);
        double best = -1.0;
        for (size_t i = 0; i < geo.sx.size(); ++i)
            if (geo.sx[i] >= x0 && geo.sx[i] <= x1 && geo.sy[i] >= y0 && geo.sy[i] <= y1) {
                double L = geo.plen[geo.spanel[i]];
                if (best < 0 || L < best) best = L;
            }
        return best;
    }

    // Phase-A split decisions for one level's frontier
    std::vector<uint8_t> decide(const std::vector<uint64_t> &front) {
        std::vector<uint8_t> split(front.size(), 0);
        std::vector<size_t> eval;
        for (size_t i = 0; i < front.size(); ++i) {
            int l = key_level(front[i]);
            if (l >= opt.max_level) continue;
            if (l < opt.min_level) {
                split[i] = 1;
                continue;
            }
            if (opt.refine_tol <= 0.0) continue;
            eval.push_back(i);
        }
        if (eval.empty()) return split;
        std::vector<uint64_t> ks;
        for (size_t i : eval) ks.push_back(front[i]);
        classify(ks);
        std::vector<size_t> need_f;
        for (size_t i : eval) {
            int c = cls[front[i]];
            if (c == kExterior) continue;
            if (c == kCut) {
                double L = min_panel_len_in(front[i]);
                double side = std::ldexp(1.0, -key_level(front[i]));
                if (L > 0 && side > 2.0 * L) {
                    split[i] = 1;
                    continue;
                }
            }
            need_f.push_back(i);
        }
        if (need_f.empty()) return split;
        const int K = opt.K, KK = K * K;
        std::vector<double> xy(2 * (size_t)KK * need_f.size()), fv((size_t)KK * need_f.size());
        for (size_t n = 0; n < need_f.size(); ++n) nodes_of(front[need_f[n]], xy.data() + 2 * KK * n);
        if (cb.f(xy.data(), (int64_t)fv.size(), fv.data(), cb.ctx) != 0)
            fail(VPX_ERR_CALLBACK, "f callback failed");
        const double thr = opt.refine_tol * opt.f_scale;
        std::vector<double> tmp(KK);
        for (size_t n = 0; n < need_f.size(); ++n) {
            const double *F = fv.data() + KK * n;   // F[b*K + a]
            // Legendre coefficients by Gauss quadrature:
            // c_mn = (2m+1)(2n+1)/4 sum_ab w_a w_b P_m(t_a) P_n(t_b) F_ab
            for (int b = 0; b < K; ++b)
                for (int m = 0; m < K; ++m) {
                    double s = 0.0;
                    for (int a = 0; a < K; ++a) s += tw[a] * Pm[m * K + a] * F[b * K + a];
                    tmp[b * K + m] = s;
                }
            double tail = 0.0;
            for (int nn = 0; nn < K; ++nn)
                for (int m = 0; m < K; ++m) {
                    if (m + nn < K - 1) continue;
                    double s = 0.0;
                    for (int b = 0; b < K; ++b) s += tw[b] * Pm[nn * K + b] * tmp[b * K + m];
                    s *= (2 * m + 1) * (2 * nn + 1) * 0.25;
                    tail = std::max(tail, std::fabs(s));
                }
            if (tail > thr) split[need_f[n]] = 1;
        }
        return split;
    }
};

}  // namespace

void build_tree(const vpx_options &opt, const Callbacks &cb, HostTree &tree) {
    Builder B(opt, cb);
    std::unordered_set<uint64_t> leaves;
    std::vector<uint64_t> front{box_key(0, 0, 0)};
    while (!front.empty()) {
        std::vector<uint8_t> sp = B.decide(front);
        std::vector<uint64_t> nxt;
        for (size_t i = 0; i < front.size(); ++i) {
            if (sp[i]) {
                if (key_level(front[i]) + 1 > kMaxLevel) fail(VPX_ERR_LEVEL, "maximum level exceeded");
                for (int c = 0; c < 4; ++c) nxt.push_back(child_key(front[i], c));
            } else {
                leaves.insert(front[i]);
            }
        }
        front.swap(nxt);
    }

    auto leaf_containing = [&](uint64_t p) -> int64_t {
        for (int lev = key_level(p); lev >= 0; --lev) {
            uint64_t a = ancestor_key(p, lev);
            if (leaves.count(a)) return (int64_t)a;
        }
        return -1;
    };
    auto split_leaf = [&](uint64_t k) {
        if (key_level(k) + 1 > kMaxLevel) fail(VPX_ERR_LEVEL, "maximum level exceeded");
        leaves.erase(k);
        for (int c = 0; c < 4; ++c) leaves.insert(child_key(k, c));
    };
    auto neighbours = [&](uint64_t k, uint64_t *out) {
        int l = key_level(k), ix = key_ix(k), iy = key_iy(k), n = 1 << l, cnt = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                int jx = ix + dx, jy = iy + dy;
                if (jx >= 0 && jy >= 0 && jx < n && jy < n) out[cnt++] = box_key(l, jx, jy);
            }
        return cnt;
    };

    for (;;) {
        bool changed = false;
        for (;;) {   // 2:1 balance
            std::unordered_set<uint64_t> marks;
            uint64_t nb[8];
            for (uint64_t k : leaves) {
                int cnt = neighbours(k, nb);
                for (int i = 0; i < cnt; ++i) {
                    int64_t c = leaf_containing(nb[i]);
                    if (c >= 0 && key_level((uint64_t)c) < key_level(k) - 1) marks.insert((uint64_t)c);
                }
            }
            if (marks.empty()) break;
            for (uint64_t c : marks) split_leaf(c);
            changed = true;
        }
        // extension restriction
        std::vector<uint64_t> all(leaves.begin(), leaves.end());
        B.classify(all);
        std::unordered_set<uint64_t> marks;
        uint64_t nb[8];
        for (uint64_t k : all) {
            if (B.cls[k] != kCut) continue;
            int cnt = neighbours(k, nb);
            for (int i = 0; i < cnt; ++i) {
                int64_t c = leaf_containing(nb[i]);
                if (c >= 0 && key_level((uint64_t)c) < key_level(k) && B.cls[(uint64_t)c] == kExterior)
                    marks.insert((uint64_t)c);
            }
        }
        if (!marks.empty()) {
            for (uint64_t c : marks) split_leaf(c);
            changed = true;
        }
        if (!changed) break;
    }

    std::vector<uint64_t> all(leaves.begin(), leaves.end());
    B.classify(all);
    int lmax = 0;
    for (uint64_t k : all) lmax = std::max(lmax, key_level(k));
    auto zkey = [&](uint64_t k) {
        int sh = lmax - key_level(k);
        return (uint64_t)morton2((uint32_t)key_ix(k) << sh, (uint32_t)key_iy(k) << sh);
    };
    std::sort(all.begin(), all.end(), [&](uint64_t a, uint64_t b) { return zkey(a) < zkey(b); });

    tree.K = opt.K;
    tree.max_level = lmax;
    tree.leaves.resize(all.size());
    std::unordered_map<uint64_t, int32_t> index;
    for (size_t i = 0; i < all.size(); ++i) {
        uint64_t k = all[i];
        tree.leaves[i] = Leaf{key_level(k), key_ix(k), key_iy(k), B.cls[k], -1};
        index[k] = (int32_t)i;
        if (B.cls[k] == kCut) {
            int l = key_level(k), n = 1 << l;
            if (key_ix(k) < 1 || key_iy(k) < 1 || key_ix(k) > n - 2 || key_iy(k) > n - 2)
                fail(VPX_ERR_DOMAIN, "extension square of a cut leaf leaves D");
        }
    }
    // extension lists: owner of each exterior leaf
    for (size_t i = 0; i < all.size(); ++i) {
        if (tree.leaves[i].cls != kExterior) continue;
        const Leaf &L = tree.leaves[i];
        double x0, x1, y0, y1;
        box_bounds(all[i], x0, x1, y0, y1);
        double cx = 0.5 * (x0 + x1), cy = 0.5 * (y0 + y1);
        int32_t best = -1;
        double bestd = 0.0;
        for (int lev = 0; lev <= L.level; ++lev) {
            int ax = L.ix >> (L.level - lev), ay = L.iy >> (L.level - lev), n = 1 << lev;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int sx = ax + dx, sy = ay + dy;
                    if (sx < 0 || sy < 0 || sx >= n || sy >= n) continue;
                    auto it = index.find(box_key(lev, sx, sy));
                    if (it == index.end()) continue;
                    int32_t j = it->second;
                    if (tree.leaves[j].cls != kCut) continue;
                    double s = std::ldexp(1.0, -lev);
                    double scx = -0.5 + (sx + 0.5) * s, scy = -0.5 + (sy + 0.5) * s;
                    double d = (scx - cx) * (scx - cx) + (scy - cy) * (scy - cy);
                    if (best < 0 || d < bestd || (d == bestd && j > best)) {
                        best = j;
                        bestd = d;
                    }
                }
        }
        tree.leaves[i].owner = best;
    }
}

}  // namespace vpx
