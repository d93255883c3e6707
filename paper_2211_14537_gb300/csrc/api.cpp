// api.cpp -- the extern "C" entry points declared in include/vpx.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>

#include "lists.h"
#include "plan.h"

namespace vpx {

static thread_local std::string g_last_error;

void set_error_message(const std::string &m) { g_last_error = m; }

void fail(int code, const std::string &m) { throw Error{code, m}; }

template <class F>
static int guarded(F &&f) {
    try {
        f();
        return VPX_OK;
    } catch (const Error &e) {
        set_error_message(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error_message("host allocation failed");
        return VPX_ERR_NOMEM;
    } catch (...) {
        set_error_message("unexpected exception");
        return VPX_ERR_ARG;
    }
}

// All boxes (leaves and their ancestors), sorted by level then Morton key.
void build_boxes(vpx_plan *p) {
    const auto &L = p->tree.leaves;
    std::vector<uint64_t> keys;
    std::unordered_map<uint64_t, int32_t> leaf_of;
    for (size_t i = 0; i < L.size(); ++i) {
        uint64_t k = box_key(L[i].level, L[i].ix, L[i].iy);
        leaf_of[k] = (int32_t)i;
        for (int lev = L[i].level; lev >= 0; --lev)
            keys.push_back(box_key(lev, L[i].ix >> (L[i].level - lev), L[i].iy >> (L[i].level - lev)));
    }
    std::sort(keys.begin(), keys.end(), [](uint64_t a, uint64_t b) {
        int la = key_level(a), lb = key_level(b);
        if (la != lb) return la < lb;
        return morton2(key_ix(a), key_iy(a)) < morton2(key_ix(b), key_iy(b));
    });
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    const int nb = (int)keys.size();
    p->n_levels = p->tree.max_level + 1;
    p->box_level.resize(nb);
    p->box_ix.resize(nb);
    p->box_iy.resize(nb);
    p->box_parent.assign(nb, -1);
    p->box_child0.assign(nb, -1);
    p->box_leaf.assign(nb, -1);
    p->box_morton.resize(nb);
    std::unordered_map<uint64_t, int32_t> idx;
    for (int b = 0; b < nb; ++b) {
        uint64_t k = keys[b];
        p->box_level[b] = key_level(k);
        p->box_ix[b] = key_ix(k);
        p->box_iy[b] = key_iy(k);
        p->box_morton[b] = morton2(key_ix(k), key_iy(k));
        idx[k] = b;
        auto it = leaf_of.find(k);
        if (it != leaf_of.end()) p->box_leaf[b] = it->second;
    }
    std::fill(p->level_start, p->level_start + kMaxLevel + 2, nb);
    for (int b = nb - 1; b >= 0; --b) p->level_start[p->box_level[b]] = b;
    for (int l = kMaxLevel; l >= 0; --l)
        if (p->level_start[l] > p->level_start[l + 1]) p->level_start[l] = p->level_start[l + 1];
    p->level_start[0] = 0;
    for (int b = 0; b < nb; ++b) {
        int l = p->box_level[b];
        if (l > 0) {
            int par = idx[box_key(l - 1, p->box_ix[b] >> 1, p->box_iy[b] >> 1)];
            p->box_parent[b] = par;
            if ((p->box_ix[b] & 1) == 0 && (p->box_iy[b] & 1) == 0) p->box_child0[par] = b;
        }
    }
    p->leaf_nz.assign(L.size(), 0);
    for (size_t i = 0; i < L.size(); ++i) p->leaf_nz[i] = (L[i].cls != kExterior || L[i].owner >= 0) ? 1 : 0;
    p->box_nz.assign(nb, 0);
    for (int b = nb - 1; b >= 0; --b) {
        if (p->box_leaf[b] >= 0) p->box_nz[b] = p->leaf_nz[p->box_leaf[b]];
        if (p->box_nz[b] && p->box_parent[b] >= 0) p->box_nz[p->box_parent[b]] = 1;
    }
}

static ListView host_view(vpx_plan *p) {
    ListView v;
    v.n_levels = p->n_levels;
    v.level_start = p->level_start;
    v.morton = p->box_morton.data();
    v.box_level = p->box_level.data();
    v.box_ix = p->box_ix.data();
    v.box_iy = p->box_iy.data();
    v.box_child0 = p->box_child0.data();
    v.box_leaf = p->box_leaf.data();
    v.box_nz = p->box_nz.data();
    v.leaf_nz = p->leaf_nz.data();
    return v;
}

void build_lists_host(vpx_plan *p) {
    const int nb = (int)p->box_level.size(), nl = (int)p->tree.leaves.size();
    p->near.assign((size_t)nl * kNearConfigs, -1);
    p->vlist.assign((size_t)nb * kVSlots, -1);
    p->xlist.assign((size_t)nb * kXSlots, -1);
    p->wlist.assign((size_t)nl * kWSlots, -1);
    ListView v = host_view(p);
    for (int b = 0; b < nb; ++b) {
        int lf = p->box_leaf[b];
        lv_build_box(v, b, lf >= 0 ? &p->near[(size_t)lf * kNearConfigs] : nullptr, &p->vlist[(size_t)b * kVSlots],
                     &p->xlist[(size_t)b * kXSlots], lf >= 0 ? &p->wlist[(size_t)lf * kWSlots] : nullptr);
    }
}

static void count_lists(vpx_plan *p) {
    auto cnt = [](const std::vector<int32_t> &a) {
        int64_t c = 0;
        for (int32_t x : a) c += (x >= 0);
        return c;
    };
    p->cnt_near = cnt(p->near);
    p->cnt_m2l = cnt(p->vlist);
    p->cnt_s2l = cnt(p->xlist);
    p->cnt_m2t = cnt(p->wlist);
}

static void build_leaf_and_boundary_nodes(vpx_plan *p, const Callbacks &cb) {
    const int K = p->K;
    std::vector<double> t, tw;
    gauss_legendre(K, t, tw);
    const auto &L = p->tree.leaves;
    p->leaf_xy.resize(2 * L.size() * K * K);
    for (size_t i = 0; i < L.size(); ++i) {
        double s = std::ldexp(1.0, -L[i].level), h = 0.5 * s;
        double cx = -0.5 + (L[i].ix + 0.5) * s, cy = -0.5 + (L[i].iy + 0.5) * s;
        for (int b = 0; b < K; ++b)
            for (int a = 0; a < K; ++a) {
                p->leaf_xy[2 * (i * K * K + b * K + a)] = cx + h * t[a];
                p->leaf_xy[2 * (i * K * K + b * K + a) + 1] = cy + h * t[b];
            }
    }
    const int nq = p->opt.n_quad_bdry;
    std::vector<double> g, gw;
    gauss_legendre(nq, g, gw);
    p->bdry_xy.resize(2 * (size_t)cb.n_panels * nq);
    p->bdry_dxy.resize(2 * (size_t)cb.n_panels * nq);
    p->bdry_ends.resize(4 * (size_t)cb.n_panels);
    const double ends_t[2] = {-1.0, 1.0};
    double ends_d[4];
    for (int i = 0; i < cb.n_panels; ++i) {
        if (cb.curve(i, g.data(), nq, &p->bdry_xy[2 * (size_t)i * nq], &p->bdry_dxy[2 * (size_t)i * nq], cb.ctx) != 0 ||
            cb.curve(i, ends_t, 2, &p->bdry_ends[4 * (size_t)i], ends_d, cb.ctx) != 0)
            fail(VPX_ERR_CALLBACK, "curve callback failed");
    }
    // containing leaf (a point on an edge belongs to the box with the larger
    // index, except on the top/right edge of D) and its Lagrange weights
    std::unordered_map<uint64_t, int32_t> idx;
    for (size_t i = 0; i < L.size(); ++i) idx[box_key(L[i].level, L[i].ix, L[i].iy)] = (int32_t)i;
    std::vector<double> bw = barycentric_weights(t);
    const size_t nbd = p->bdry_xy.size() / 2;
    p->bdry_leaf.assign(nbd, -1);
    p->bdry_w.assign(nbd * 2 * K, 0.0);
    for (size_t k = 0; k < nbd; ++k) {
        double x = p->bdry_xy[2 * k], y = p->bdry_xy[2 * k + 1];
        if (!(x >= -0.5 && x <= 0.5 && y >= -0.5 && y <= 0.5)) fail(VPX_ERR_DOMAIN, "boundary node outside D");
        int32_t found = -1;
        for (int lev = 0; lev <= p->tree.max_level && found < 0; ++lev) {
            int n = 1 << lev;
            int ix = std::min((int)std::floor((x + 0.5) * n), n - 1);
            int iy = std::min((int)std::floor((y + 0.5) * n), n - 1);
            auto it = idx.find(box_key(lev, ix, iy));
            if (it != idx.end()) found = it->second;
        }
        if (found < 0) fail(VPX_ERR_DOMAIN, "boundary node not in any leaf");
        p->bdry_leaf[k] = found;
        const Leaf &lf = L[found];
        double s = std::ldexp(1.0, -lf.level), h = 0.5 * s;
        double cx = -0.5 + (lf.ix + 0.5) * s, cy = -0.5 + (lf.iy + 0.5) * s;
        lagrange_eval(t, bw, (x - cx) / h, &p->bdry_w[k * 2 * K]);
        lagrange_eval(t, bw, (y - cy) / h, &p->bdry_w[k * 2 * K + K]);
    }
}

static void check_options(const vpx_options *o) {
    if (!o) fail(VPX_ERR_ARG, "null options");
    if (o->K < 4 || o->K > kMaxK || (o->K % 2)) fail(VPX_ERR_ARG, "K must be even, 4..16");
    if (o->min_level < 0 || o->max_level > kMaxLevel || o->min_level > o->max_level)
        fail(VPX_ERR_ARG, "levels must satisfy 0 <= min_level <= max_level <= 15");
    if (o->p < 8 || o->p + 1 > kMaxP) fail(VPX_ERR_ARG, "p must be in 8..63");
    if (o->refine_tol < 0 || !(o->f_scale > 0)) fail(VPX_ERR_ARG, "refine_tol >= 0 and f_scale > 0 required");
    if (o->precision != VPX_PREC_FP64 && o->precision != VPX_PREC_MIXED) fail(VPX_ERR_ARG, "bad precision");
    if (o->max_rhs < 1) fail(VPX_ERR_ARG, "max_rhs >= 1 required");
    if (o->n_quad_bdry < 1 || o->n_quad_bdry > 64) fail(VPX_ERR_ARG, "n_quad_bdry in 1..64");
    check_rbf_eps(o->K, o->rbf_eps);
    if (o->ext_mode != 0 && o->ext_mode != 1) fail(VPX_ERR_ARG, "ext_mode must be 0 or 1");
    if (o->ext_mode == 1 && o->rbf_eps != 0.0) fail(VPX_ERR_ARG, "rbf_eps applies to the universal stencil only");
}

}  // namespace vpx

using namespace vpx;

extern "C" {

int vpx_universal_matrix(int K, double rbf_eps, double *out, int64_t *nx, int64_t *ng) {
    return guarded([&] {
        if (!nx || !ng) fail(VPX_ERR_ARG, "null size pointer");
        if (K < 4 || K > kMaxK || (K % 2)) fail(VPX_ERR_ARG, "K must be even, 4..16");
        check_rbf_eps(K, rbf_eps);
        std::vector<double> A;
        int NX = 0, NG = 0;
        universal_operator(K, rbf_eps, A, NX, NG);
        *nx = NX;
        *ng = NG;
        if (out) std::copy(A.begin(), A.end(), out);
    });
}

int vpx_plan_ray_operator(vpx_plan_t p, int64_t *n_ray, int32_t *ray_c, int32_t *ray_g, int64_t *ray_src,
                          double *coef) {
    return guarded([&] {
        if (!p || !n_ray) fail(VPX_ERR_ARG, "null argument");
        const StencilInfo &st = p->st;
        if (st.mode != 1) fail(VPX_ERR_STATE, "the plan extends with the universal stencil");
        *n_ray = (int64_t)st.ray_c.size();
        if (ray_c) std::copy(st.ray_c.begin(), st.ray_c.end(), ray_c);
        if (ray_g) std::copy(st.ray_g.begin(), st.ray_g.end(), ray_g);
        if (ray_src) std::copy(st.ray_src.begin(), st.ray_src.end(), ray_src);
        if (coef) std::copy(st.ray_coef.begin(), st.ray_coef.end(), coef);
    });
}

int vpx_default_options(vpx_options *opt) {
    if (!opt) return VPX_ERR_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->K = 8;
    opt->min_level = 4;
    opt->max_level = 4;
    opt->refine_tol = 0.0;
    opt->f_scale = 1.0;
    opt->p = 44;
    opt->precision = VPX_PREC_FP64;
    opt->max_rhs = 1;
    opt->n_quad_bdry = 16;
    return VPX_OK;
}

int vpx_plan_create(const vpx_options *opt, int n_panels, vpx_curve_cb curve, vpx_inside_cb inside,
                    vpx_points_cb refine_f, void *ctx, unsigned flags, vpx_plan_t *out) {
    if (!out) return VPX_ERR_ARG;
    *out = nullptr;
    vpx_plan *p = nullptr;
    int rc = guarded([&] {
        check_options(opt);
        if (n_panels < 0 || (n_panels > 0 && !curve) || !inside || !refine_f)
            fail(VPX_ERR_ARG, "missing callback");
        p = new vpx_plan();
        static std::atomic<uint64_t> next_uid{1};
        p->uid = next_uid++;
        p->opt = *opt;
        p->host_only = (flags & VPX_PLAN_HOST_ONLY) != 0;
        p->K = opt->K;
        p->KK = opt->K * opt->K;
        p->P = opt->p + 1;
        Callbacks cb{curve, inside, refine_f, ctx, n_panels};
        build_tree(p->opt, cb, p->tree);
        build_stencil(p->opt, cb, p->tree, p->stencil_xy, p->st, !p->host_only);
        build_leaf_and_boundary_nodes(p, cb);
        build_boxes(p);
        if (p->host_only)
            build_lists_host(p);
        else
            device_setup(p);   // builds the interaction lists on the device
        count_lists(p);
    });
    if (rc != VPX_OK) {
        if (p) {
            if (!p->host_only) device_free(p);
            delete p;
        }
        return rc;
    }
    *out = p;
    return VPX_OK;
}

int vpx_plan_sizes(vpx_plan_t p, int64_t *n_leaves, int64_t *n_leaf_nodes, int64_t *n_stencil, int64_t *n_bdry) {
    if (!p) return VPX_ERR_ARG;
    if (n_leaves) *n_leaves = (int64_t)p->tree.leaves.size();
    if (n_leaf_nodes) *n_leaf_nodes = (int64_t)p->tree.leaves.size() * p->KK;
    if (n_stencil) *n_stencil = (int64_t)p->stencil_xy.size() / 2;
    if (n_bdry) *n_bdry = (int64_t)p->bdry_xy.size() / 2;
    return VPX_OK;
}

int vpx_plan_leaves(vpx_plan_t p, int32_t *level, int32_t *ix, int32_t *iy, int32_t *cls, int32_t *owner) {
    if (!p) return VPX_ERR_ARG;
    const auto &L = p->tree.leaves;
    for (size_t i = 0; i < L.size(); ++i) {
        if (level) level[i] = L[i].level;
        if (ix) ix[i] = L[i].ix;
        if (iy) iy[i] = L[i].iy;
        if (cls) cls[i] = L[i].cls;
        if (owner) owner[i] = L[i].owner;
    }
    return VPX_OK;
}

int vpx_stencil_points(vpx_plan_t p, double *xy) {
    if (!p || !xy) return VPX_ERR_ARG;
    std::copy(p->stencil_xy.begin(), p->stencil_xy.end(), xy);
    return VPX_OK;
}

int vpx_leaf_nodes(vpx_plan_t p, double *xy) {
    if (!p || !xy) return VPX_ERR_ARG;
    std::copy(p->leaf_xy.begin(), p->leaf_xy.end(), xy);
    return VPX_OK;
}

int vpx_boundary_nodes(vpx_plan_t p, double *xy) {
    if (!p || !xy) return VPX_ERR_ARG;
    std::copy(p->bdry_xy.begin(), p->bdry_xy.end(), xy);
    return VPX_OK;
}

int vpx_plan_list_counts(vpx_plan_t p, int64_t *near, int64_t *m2l, int64_t *s2l, int64_t *m2t, int64_t *n_boxes,
                         int32_t *n_levels) {
    if (!p) return VPX_ERR_ARG;
    if (near) *near = p->cnt_near;
    if (m2l) *m2l = p->cnt_m2l;
    if (s2l) *s2l = p->cnt_s2l;
    if (m2t) *m2t = p->cnt_m2t;
    if (n_boxes) *n_boxes = (int64_t)p->box_level.size();
    if (n_levels) *n_levels = p->n_levels;
    return VPX_OK;
}

// Host copies of the fixed-slot lists (for tests): sizes n_leaves*33, n_boxes*40,
// n_boxes*20, n_leaves*20, and the boxes (level, ix, iy, leaf) of length n_boxes.
int vpx_plan_lists(vpx_plan_t p, int32_t *near, int32_t *vlist, int32_t *xlist, int32_t *wlist, int32_t *box_level,
                   int32_t *box_ix, int32_t *box_iy, int32_t *box_leaf) {
    if (!p) return VPX_ERR_ARG;
    if (near) std::copy(p->near.begin(), p->near.end(), near);
    if (vlist) std::copy(p->vlist.begin(), p->vlist.end(), vlist);
    if (xlist) std::copy(p->xlist.begin(), p->xlist.end(), xlist);
    if (wlist) std::copy(p->wlist.begin(), p->wlist.end(), wlist);
    if (box_level) std::copy(p->box_level.begin(), p->box_level.end(), box_level);
    if (box_ix) std::copy(p->box_ix.begin(), p->box_ix.end(), box_ix);
    if (box_iy) std::copy(p->box_iy.begin(), p->box_iy.end(), box_iy);
    if (box_leaf) std::copy(p->box_leaf.begin(), p->box_leaf.end(), box_leaf);
    return VPX_OK;
}

int vpx_plan_near_tables(vpx_plan_t p, double *out) {
    return guarded([&] {
        if (!p || !out) fail(VPX_ERR_ARG, "null argument");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        device_copy_near_tables(p, out);
    });
}

int vpx_execute(vpx_plan_t p, const double *f, int nrhs, int64_t ld_f, double *v, int64_t ld_v, double *vb,
                int64_t ld_b, void *stream) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        int64_t ns = (int64_t)p->stencil_xy.size() / 2, nt = (int64_t)p->leaf_xy.size() / 2;
        int64_t nbd = (int64_t)p->bdry_xy.size() / 2;
        if (nrhs < 1 || nrhs > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range");
        if ((ns && !f) || !v || ld_f < ns || ld_v < nt || (vb && ld_b < nbd)) fail(VPX_ERR_ARG, "bad buffer");
        device_execute(p, f, nrhs, ld_f, v, ld_v, vb, ld_b, stream);
    });
}

int vpx_execute_batch(int n, vpx_plan_t const *plans, const double *const *f, const int *nrhs, const int64_t *ld_f,
                      double *const *v, const int64_t *ld_v, double *const *vb, const int64_t *ld_b, void *stream) {
    return guarded([&] {
        if (n < 1 || !plans || !f || !nrhs || !ld_f || !v || !ld_v || !vb || !ld_b) fail(VPX_ERR_ARG, "null batch array");
        for (int i = 0; i < n; ++i) {
            vpx_plan *p = plans[i];
            if (!p) fail(VPX_ERR_ARG, "null plan in batch");
            for (int j = 0; j < i; ++j)
                if (plans[j] == p) fail(VPX_ERR_ARG, "a plan appears twice in a batch");
            int64_t ns = (int64_t)p->stencil_xy.size() / 2, nt = (int64_t)p->leaf_xy.size() / 2;
            int64_t nbd = (int64_t)p->bdry_xy.size() / 2;
            if (nrhs[i] < 1 || nrhs[i] > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range in batch");
            if ((ns && !f[i]) || !v[i] || ld_f[i] < ns || ld_v[i] < nt || (vb[i] && ld_b[i] < nbd))
                fail(VPX_ERR_ARG, "bad buffer in batch");
        }
        for (int i = 0; i < n; ++i)
            if (plans[i]->host_only) fail(VPX_ERR_STATE, "host-only plan in batch");
        device_execute_batch(n, plans, f, nrhs, ld_f, v, ld_v, vb, ld_b, stream);
    });
}

int vpx_autotune(vpx_plan_t p, const double *f, int nrhs, int64_t ld_f, void *stream, int *n_passes, int *n_changed) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        const int64_t ns = (int64_t)p->stencil_xy.size() / 2;
        if (nrhs < 1 || nrhs > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range");
        if ((ns && !f) || ld_f < ns) fail(VPX_ERR_ARG, "bad stencil buffer");
        device_autotune(1, &p, &f, &nrhs, &ld_f, stream, n_passes, n_changed);
    });
}

int vpx_autotune_batch(int n, vpx_plan_t const *plans, const double *const *f, const int *nrhs, const int64_t *ld_f,
                       void *stream, int *n_passes, int *n_changed) {
    return guarded([&] {
        if (n < 1 || !plans || !f || !nrhs || !ld_f) fail(VPX_ERR_ARG, "null batch array");
        for (int i = 0; i < n; ++i) {
            vpx_plan *p = plans[i];
            if (!p) fail(VPX_ERR_ARG, "null plan in batch");
            for (int j = 0; j < i; ++j)
                if (plans[j] == p) fail(VPX_ERR_ARG, "a plan appears twice in a batch");
            const int64_t ns = (int64_t)p->stencil_xy.size() / 2;
            if (nrhs[i] < 1 || nrhs[i] > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range in batch");
            if ((ns && !f[i]) || ld_f[i] < ns) fail(VPX_ERR_ARG, "bad stencil buffer in batch");
        }
        for (int i = 0; i < n; ++i)
            if (plans[i]->host_only) fail(VPX_ERR_STATE, "host-only plan in batch");
        device_autotune(n, plans, f, nrhs, ld_f, stream, n_passes, n_changed);
    });
}

int vpx_extend(vpx_plan_t p, const double *f, int nrhs, int64_t ld_f, double *fe, int64_t ld_fe, void *stream) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        int64_t ns = (int64_t)p->stencil_xy.size() / 2, nt = (int64_t)p->leaf_xy.size() / 2;
        if (nrhs < 1 || nrhs > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range");
        if ((ns && !f) || !fe || ld_f < ns || ld_fe < nt) fail(VPX_ERR_ARG, "bad buffer");
        device_extend(p, f, nrhs, ld_f, fe, ld_fe, stream);
    });
}

int vpx_potential(vpx_plan_t p, const double *fe, int nrhs, int64_t ld_fe, double *v, int64_t ld_v, double *vb,
                  int64_t ld_b, void *stream) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        int64_t nt = (int64_t)p->leaf_xy.size() / 2, nbd = (int64_t)p->bdry_xy.size() / 2;
        if (nrhs < 1 || nrhs > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range");
        if (!fe || !v || ld_fe < nt || ld_v < nt || (vb && ld_b < nbd)) fail(VPX_ERR_ARG, "bad buffer");
        device_potential(p, fe, ld_fe, nrhs, v, ld_v, vb, ld_b, stream);
    });
}

int vpx_potential_static(vpx_plan_t p, const double *fe, int nrhs, int64_t ld_fe, double *v, int64_t ld_v,
                         double *vb, int64_t ld_b, void *stream) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        // the slice buffers of the mixed form are plan workspace sized by max_rhs,
        // so the column count is bounded here as in vpx_potential (checked first,
        // before any device state is touched)
        if (nrhs < 1 || nrhs > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        int64_t nt = (int64_t)p->leaf_xy.size() / 2, nbd = (int64_t)p->bdry_xy.size() / 2;
        if (!fe || !v || ld_fe < nt || ld_v < nt || (vb && ld_b < nbd)) fail(VPX_ERR_ARG, "bad buffer");
        device_potential_static(p, fe, ld_fe, nrhs, v, ld_v, vb, ld_b, stream);
    });
}

int vpx_bie_setup(vpx_plan_t p, vpx_inside_cb inside, void *ctx) {
    return guarded([&] {
        if (!p || !inside) fail(VPX_ERR_ARG, "null argument");
        bie_setup(p, inside, ctx);
    });
}

int vpx_bie_topology(vpx_plan_t p, int *n_curves, int *outer_curve, int32_t *curve_of_node, double *jump) {
    return guarded([&] {
        if (!p || !n_curves || !outer_curve) fail(VPX_ERR_ARG, "null argument");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        *n_curves = p->bie.n_curves;
        *outer_curve = p->bie.outer_curve;
        if (curve_of_node) std::copy(p->bie.curve_of_node.begin(), p->bie.curve_of_node.end(), curve_of_node);
        if (jump) std::copy(p->bie.jump.begin(), p->bie.jump.end(), jump);
    });
}

int vpx_bie_log_terms(vpx_plan_t p, int *n_log, int32_t *curve, double *centre, int64_t *n_unknowns) {
    return guarded([&] {
        if (!p || !n_log || !n_unknowns) fail(VPX_ERR_ARG, "null argument");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        *n_log = p->bie.n_log;
        *n_unknowns = p->bie.n_unknowns;
        if (curve) std::copy(p->bie.log_curve.begin(), p->bie.log_curve.end(), curve);
        if (centre) std::copy(p->bie.log_centre.begin(), p->bie.log_centre.end(), centre);
    });
}

int vpx_bie_solve(vpx_plan_t p, const double *g, const double *vb, double growth, double *sol, void *stream) {
    return guarded([&] {
        if (!p || !g || !vb || !sol) fail(VPX_ERR_ARG, "null argument");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        device_bie_solve(p, g, vb, growth, sol, stream);
    });
}

int vpx_bie_eval(vpx_plan_t p, const double *sol, const double *v_leaf, double *u_leaf, void *stream) {
    return guarded([&] {
        if (!p || !sol || !v_leaf || !u_leaf) fail(VPX_ERR_ARG, "null argument");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        device_bie_eval(p, sol, v_leaf, u_leaf, stream);
    });
}

int vpx_bie_dipole_multipoles(vpx_plan_t p, int *n_coef, double *out) {
    return guarded([&] {
        if (!p || !n_coef) fail(VPX_ERR_ARG, "null argument");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        *n_coef = 2 * p->P;
        if (out) std::copy(p->bie.p2m.begin(), p->bie.p2m.end(), out);
    });
}

int vpx_bie_geometry(vpx_plan_t p, double *nu, double *sw, double *kappa) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        if (nu) std::copy(p->bie.nu.begin(), p->bie.nu.end(), nu);
        if (sw) std::copy(p->bie.sw.begin(), p->bie.sw.end(), sw);
        if (kappa) std::copy(p->bie.kappa.begin(), p->bie.kappa.end(), kappa);
    });
}

int vpx_bie_corrections(vpx_plan_t p, int64_t *n_corr, int64_t *off, int32_t *panel, double *w) {
    return guarded([&] {
        if (!p || !n_corr) fail(VPX_ERR_ARG, "null argument");
        if (!p->bie.ready) fail(VPX_ERR_STATE, "vpx_bie_setup has not run");
        *n_corr = (int64_t)p->bie.corr_panel.size();
        if (off) std::copy(p->bie.corr_off.begin(), p->bie.corr_off.end(), off);
        if (panel) std::copy(p->bie.corr_panel.begin(), p->bie.corr_panel.end(), panel);
        if (w) std::copy(p->bie.corr_w.begin(), p->bie.corr_w.end(), w);
    });
}

int vpx_net_charge(vpx_plan_t p, const double *fe, int nrhs, int64_t ld_fe, double *charge, void *stream) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        const int64_t nt = (int64_t)p->leaf_xy.size() / 2;
        if (nrhs < 1 || nrhs > p->opt.max_rhs) fail(VPX_ERR_ARG, "nrhs out of range");
        if (!fe || !charge || ld_fe < nt) fail(VPX_ERR_ARG, "bad buffer");
        device_net_charge(p, fe, ld_fe, nrhs, charge, stream);
    });
}

int vpx_execute_host(vpx_plan_t p, const double *f, int nrhs, double *v, double *vb) {
    return guarded([&] {
        if (!p) fail(VPX_ERR_ARG, "null plan");
        if (p->host_only) fail(VPX_ERR_STATE, "host-only plan");
        if (nrhs < 1 || nrhs > p->opt.max_rhs || !v) fail(VPX_ERR_ARG, "bad argument");
        device_execute_host(p, f, nrhs, v, vb);
    });
}

int vpx_sync_status(vpx_plan_t p) {
    if (!p) return VPX_ERR_ARG;
    if (p->host_only) return VPX_OK;
    int st = VPX_OK;
    int rc = guarded([&] { st = device_sync_status(p); });
    return rc != VPX_OK ? rc : st;
}

int vpx_set_timing(vpx_plan_t p, int enable) {
    if (!p) return VPX_ERR_ARG;
    p->timing = enable != 0;
    return VPX_OK;
}

int vpx_get_timings(vpx_plan_t p, double *ms, int n) {
    if (!p || !ms || n < 0) return VPX_ERR_ARG;
    for (int i = 0; i < n && i < VPX_N_PASSES; ++i) ms[i] = p->pass_ms[i];
    return VPX_OK;
}

int vpx_check_bounded_wait(int *status) {
    if (!status) return VPX_ERR_ARG;
    return guarded([&] { return vpx::device_check_bounded_wait(status); });
}

int vpx_check_gauss_jordan(int n, const double *a, double *inv, int *status) {
    if (n < 1 || !a || !inv || !status) return VPX_ERR_ARG;
    return guarded([&] { *status = vpx::device_check_gauss_jordan(n, a, inv); });
}

int vpx_graph_kernel_count(vpx_plan_t p, int64_t *kernels) {
    if (!p || !kernels) return VPX_ERR_ARG;
    *kernels = p->graph_kernels;
    return VPX_OK;
}

const char *vpx_pass_name(int i) {
    static const char *names[VPX_N_PASSES] = {"extension", "l2m", "m2m", "m2l_s2l", "l2l",
                                              "l2t_const", "near", "join_boundary"};
    return (i >= 0 && i < VPX_N_PASSES) ? names[i] : "";
}

const char *vpx_error_string(int code) {
    switch (code) {
        case VPX_OK: return "ok";
        case VPX_ERR_ARG: return "invalid argument";
        case VPX_ERR_CUDA: return "CUDA error";
        case VPX_ERR_NOMEM: return "out of memory";
        case VPX_ERR_STENCIL: return "extension stencil cannot be formed";
        case VPX_ERR_DOMAIN: return "geometry outside the root box";
        case VPX_ERR_LEVEL: return "maximum level exceeded";
        case VPX_ERR_TIMEOUT: return "device wait timed out";
        case VPX_ERR_NAN: return "non-finite value";
        case VPX_ERR_CALLBACK: return "callback failed";
        case VPX_ERR_STATE: return "invalid plan state";
        case VPX_ERR_NODEV: return "no CUDA device";
        default: return "unknown error";
    }
}

const char *vpx_last_error_message(void) { return g_last_error.c_str(); }

void vpx_plan_destroy(vpx_plan_t p) {
    if (!p) return;
    if (!p->host_only) {
        try {
            device_free(p);
        } catch (...) {
        }
    }
    delete p;
}

}  // extern "C"
