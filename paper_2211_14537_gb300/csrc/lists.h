// lists.h -- interaction lists of the adaptive box FMM, one box at a time.
//
// Built on the host once per geometry (milliseconds for 1e5 boxes) and
// uploaded; the passes only read the resulting slot arrays.
//
// For a box B at level l (Section 4, Fig. tree_levels):
//  - near list (leaves only): colleagues that are leaves (incl. B itself),
//    coarse neighbours (leaves at level l-1 touching B) and fine neighbours
//    (leaves at level l+1 touching B); each occupies the slot of its unique
//    relative configuration (9 + 12 + 12 = 33);
//  - list i (l >= 2): children of the colleagues of B's parent that do not
//    touch B, in the slot of their offset (dx, dy) in [-3,3]^2 \ [-1,1]^2;
//  - list i+ (l >= 2): leaves at level l-1 that are colleagues of B's parent
//    and do not touch B (their sources reach B through a local expansion);
//  - list i- (leaves only): children of B's colleagues that do not touch B
//    (their multipoles are evaluated directly at B's nodes).
// Only sources with non-zero data are listed.
#pragma once

#include <cstdint>

namespace vpx {

struct ListView {
    int n_levels;
    const int32_t *level_start;   // [n_levels+1]
    const uint32_t *morton;       // per box, sorted within each level
    const int32_t *box_level, *box_ix, *box_iy, *box_child0, *box_leaf;
    const uint8_t *box_nz, *leaf_nz;
};

inline uint32_t lv_morton(uint32_t ix, uint32_t iy) {
    uint32_t k = 0;
    for (int b = 0; b < 16; ++b) {
        k |= ((ix >> b) & 1u) << (2 * b);
        k |= ((iy >> b) & 1u) << (2 * b + 1);
    }
    return k;
}

// box index at (level, ix, iy) or -1
inline int32_t lv_find(const ListView &v, int l, int ix, int iy) {
    if (l < 0 || l >= v.n_levels) return -1;
    int n = 1 << l;
    if (ix < 0 || iy < 0 || ix >= n || iy >= n) return -1;
    uint32_t key = lv_morton((uint32_t)ix, (uint32_t)iy);
    int lo = v.level_start[l], hi = v.level_start[l + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        uint32_t m = v.morton[mid];
        if (m == key) return mid;
        if (m < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// index (0..11) of position (rx, ry) in {-1,0,1,2}^2 \ {0,1}^2, row-major
inline int lv_ring12(int rx, int ry) {
    int idx = 0;
    for (int y = -1; y <= 2; ++y)
        for (int x = -1; x <= 2; ++x) {
            if (x >= 0 && x <= 1 && y >= 0 && y <= 1) continue;
            if (x == rx && y == ry) return idx;
            ++idx;
        }
    return -1;
}

// index (0..19) of position (rx, ry) in {-2..3}^2 \ {-1..2}^2, row-major
inline int lv_ring20(int rx, int ry) {
    int idx = 0;
    for (int y = -2; y <= 3; ++y)
        for (int x = -2; x <= 3; ++x) {
            if (x >= -1 && x <= 2 && y >= -1 && y <= 2) continue;
            if (x == rx && y == ry) return idx;
            ++idx;
        }
    return -1;
}

// index (0..39) of offset (dx, dy) in [-3,3]^2 \ [-1,1]^2, row-major
inline int lv_ring40(int dx, int dy) {
    int idx = 0;
    for (int y = -3; y <= 3; ++y)
        for (int x = -3; x <= 3; ++x) {
            if (x >= -1 && x <= 1 && y >= -1 && y <= 1) continue;
            if (x == dx && y == dy) return idx;
            ++idx;
        }
    return -1;
}

inline bool lv_touch(int l1, int x1, int y1, int l2, int x2, int y2) {
    // closed boxes touch: compare on the finer grid
    int L = l1 > l2 ? l1 : l2;
    int a0 = x1 << (L - l1), a1 = (x1 + 1) << (L - l1), b0 = x2 << (L - l2), b1 = (x2 + 1) << (L - l2);
    int c0 = y1 << (L - l1), c1 = (y1 + 1) << (L - l1), d0 = y2 << (L - l2), d1 = (y2 + 1) << (L - l2);
    return a0 <= b1 && b0 <= a1 && c0 <= d1 && d0 <= c1;
}

inline void lv_build_box(const ListView &v, int b, int32_t *near /*33 or null*/, int32_t *vl /*40*/,
                                int32_t *xl /*20*/, int32_t *wl /*20 or null*/) {
    const int l = v.box_level[b], ix = v.box_ix[b], iy = v.box_iy[b];
    const int leaf = v.box_leaf[b];
    for (int s = 0; s < 40; ++s) vl[s] = -1;
    for (int s = 0; s < 20; ++s) xl[s] = -1;
    if (near)
        for (int s = 0; s < 33; ++s) near[s] = -1;
    if (wl)
        for (int s = 0; s < 20; ++s) wl[s] = -1;
    if (leaf >= 0 && near) {
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int c = lv_find(v, l, ix + dx, iy + dy);
                int n = 1 << l;
                if (ix + dx < 0 || iy + dy < 0 || ix + dx >= n || iy + dy >= n) continue;
                if (c >= 0) {
                    int cl = v.box_leaf[c];
                    if (cl >= 0) {
                        if (v.leaf_nz[cl]) near[(dx + 1) + 3 * (dy + 1)] = cl;
                    } else {
                        // fine neighbours: children of c touching B
                        int c0 = v.box_child0[c];
                        for (int k = 0; k < 4; ++k) {
                            int ch = c0 + k;
                            int chx = v.box_ix[ch], chy = v.box_iy[ch];
                            if (!lv_touch(l, ix, iy, l + 1, chx, chy)) continue;
                            int chl = v.box_leaf[ch];
                            if (chl >= 0 && v.leaf_nz[chl]) {
                                int r = lv_ring12(chx - 2 * ix, chy - 2 * iy);
                                if (r >= 0) near[21 + r] = chl;
                            }
                        }
                    }
                } else if (l >= 1) {
                    // position covered by a coarser leaf (2:1 balance: level l-1)
                    int p = lv_find(v, l - 1, (ix + dx) >> 1, (iy + dy) >> 1);
                    if (p >= 0 && v.box_leaf[p] >= 0 && v.leaf_nz[v.box_leaf[p]]) {
                        int r = lv_ring12(ix - 2 * v.box_ix[p], iy - 2 * v.box_iy[p]);
                        if (r >= 0) near[9 + r] = v.box_leaf[p];
                    }
                }
            }
    }
    if (l >= 2) {
        int px = ix >> 1, py = iy >> 1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int c = lv_find(v, l - 1, px + dx, py + dy);
                if (c < 0) continue;
                int cl = v.box_leaf[c];
                if (cl >= 0) {
                    // list i+: a leaf colleague of the parent not touching B
                    if ((dx || dy) && v.leaf_nz[cl] && !lv_touch(l, ix, iy, l - 1, px + dx, py + dy)) {
                        int r = lv_ring20(ix - 2 * (px + dx), iy - 2 * (py + dy));
                        if (r >= 0) xl[r] = cl;
                    }
                    continue;
                }
                int c0 = v.box_child0[c];
                for (int k = 0; k < 4; ++k) {
                    int ch = c0 + k;
                    int ox = v.box_ix[ch] - ix, oy = v.box_iy[ch] - iy;
                    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1) continue;
                    if (!v.box_nz[ch]) continue;
                    int r = lv_ring40(ox, oy);
                    if (r >= 0) vl[r] = ch;
                }
            }
    }
    if (leaf >= 0 && wl) {
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                int c = lv_find(v, l, ix + dx, iy + dy);
                if (c < 0 || v.box_leaf[c] >= 0) continue;
                int c0 = v.box_child0[c];
                for (int k = 0; k < 4; ++k) {
                    int ch = c0 + k;
                    if (lv_touch(l, ix, iy, l + 1, v.box_ix[ch], v.box_iy[ch])) continue;
                    if (!v.box_nz[ch]) continue;
                    int r = lv_ring20(v.box_ix[ch] - 2 * ix, v.box_iy[ch] - 2 * iy);
                    if (r >= 0) wl[r] = ch;
                }
            }
    }
}

}  // namespace vpx
