// lists_device.cu -- the interaction lists of the adaptive box FMM (Section 4,
// the near, i, i+ and i- lists of every box), built on the device: one launch
// per level, one thread per box of that level.
//
// For a box B at level l with position (ix, iy):
//  - near list (leaves only): colleagues that are leaves (B itself included),
//    leaves one level coarser touching B and leaves one level finer touching
//    B, each in the slot of its relative configuration (9 + 12 + 12 = 33);
//  - list i (l >= 2): children of the colleagues of B's parent that do not
//    touch B, in the slot of their offset in [-3,3]^2 \ [-1,1]^2 (40);
//  - list i+ (l >= 2): leaf colleagues of B's parent that do not touch B, in
//    the slot of B's position relative to them in {-2..3}^2 \ {-1..2}^2 (20);
//  - list i- (leaves only): children of B's colleagues that do not touch B, in
//    the slot of their position relative to B in {-2..3}^2 \ {-1..2}^2 (20).
// Only sources with non-zero data (box_nz, leaf_nz) are listed; -1 = empty.
//
// The boxes are sorted by (level, Morton key), so a box is found by a binary
// search over its level's keys, capped at 32 halvings.  Every loop has a fixed
// bound, and every index read from the tree is checked against the array it
// addresses before use: a bad one latches VPX_ERR_STATE in the status word and
// the access is skipped, so a malformed tree cannot make a thread loop or read
// out of bounds.
#include "dev_common.cuh"

namespace vpx {

namespace {

struct TreeView {
    int n_boxes, n_leaves, n_levels;
    const int32_t *level_start;   // [n_levels + 1]
    const uint32_t *morton;       // per box, ascending within each level
    const int32_t *ix, *iy, *child0, *leaf;
    const uint8_t *box_nz, *leaf_nz;
    int *status;
};

// x's 16 low bits in the even bit positions
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__device__ __forceinline__ bool box_ok(const TreeView &t, int b) {
    if (b >= 0 && b < t.n_boxes) return true;
    set_status(t.status, VPX_ERR_STATE);
    return false;
}

__device__ __forceinline__ bool leaf_ok(const TreeView &t, int i) {
    if (i < t.n_leaves) return true;      // negative: not a leaf, not an error
    set_status(t.status, VPX_ERR_STATE);
    return false;
}

// the box at (l, x, y), or -1
__device__ int find_box(const TreeView &t, int l, int x, int y) {
    if (l < 0 || l >= t.n_levels) return -1;
    const int n = 1 << l;
    if (x < 0 || y < 0 || x >= n || y >= n) return -1;
    const uint32_t key = spread16((uint32_t)x) | (spread16((uint32_t)y) << 1);
    int lo = max(t.level_start[l], 0), hi = min(t.level_start[l + 1], t.n_boxes) - 1;
    for (int it = 0; it < 32 && lo <= hi; ++it) {
        const int mid = lo + ((hi - lo) >> 1);
        const uint32_t m = t.morton[mid];
        if (m == key) return mid;
        if (m < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// first of the four children of a non-leaf box, or -1 (and an error) if the
// tree does not hold them
__device__ int children_of(const TreeView &t, int c) {
    const int c0 = t.child0[c];
    if (c0 >= 0 && c0 + 3 < t.n_boxes) return c0;
    set_status(t.status, VPX_ERR_STATE);
    return -1;
}

// row-major index of (x, y) in the square ring [lo,hi]^2 \ [ilo,ihi]^2, or -1
__device__ __forceinline__ int ring_slot(int x, int y, int lo, int hi, int ilo, int ihi) {
    if (x < lo || x > hi || y < lo || y > hi) return -1;
    const bool inner_row = y >= ilo && y <= ihi;
    if (inner_row && x >= ilo && x <= ihi) return -1;
    const int side = hi - lo + 1, hole = ihi - ilo + 1;
    const int inner_rows_before = max(0, min(y, ihi + 1) - ilo);
    int cols_before = x - lo;
    if (inner_row) cols_before -= max(0, min(x, ihi + 1) - ilo);
    return (y - lo) * side - inner_rows_before * hole + cols_before;
}

// closed squares (l1, x1, y1) and (l2, x2, y2) share at least a corner
__device__ __forceinline__ bool touching(int l1, int x1, int y1, int l2, int x2, int y2) {
    const int L = max(l1, l2), s1 = L - l1, s2 = L - l2;
    const int a0 = x1 << s1, a1 = (x1 + 1) << s1, b0 = x2 << s2, b1 = (x2 + 1) << s2;
    const int c0 = y1 << s1, c1 = (y1 + 1) << s1, d0 = y2 << s2, d1 = (y2 + 1) << s2;
    return a0 <= b1 && b0 <= a1 && c0 <= d1 && d0 <= c1;
}

__global__ void __launch_bounds__(128) k_lists_level(TreeView t, int l, int32_t *near, int32_t *vlist, int32_t *xlist,
                                                     int32_t *wlist) {
    const int first = max(t.level_start[l], 0), end = min(t.level_start[l + 1], t.n_boxes);
    const int b = first + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (b >= end) return;
    const int ix = t.ix[b], iy = t.iy[b];
    const int lf = t.leaf[b];
    if (!leaf_ok(t, lf)) return;
    int32_t *vl = vlist + (int64_t)b * kVSlots, *xl = xlist + (int64_t)b * kXSlots;
    for (int s = 0; s < kVSlots; ++s) vl[s] = -1;
    for (int s = 0; s < kXSlots; ++s) xl[s] = -1;
    const int n = 1 << l;
    if (lf >= 0) {
        int32_t *nr = near + (int64_t)lf * kNearConfigs;
        for (int s = 0; s < kNearConfigs; ++s) nr[s] = -1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = ix + dx, y = iy + dy;
                if (x < 0 || y < 0 || x >= n || y >= n) continue;
                const int c = find_box(t, l, x, y);
                if (c >= 0) {
                    const int cl = t.leaf[c];
                    if (!leaf_ok(t, cl)) continue;
                    if (cl >= 0) {
                        if (t.leaf_nz[cl]) nr[(dx + 1) + 3 * (dy + 1)] = cl;
                        continue;
                    }
                    const int c0 = children_of(t, c);       // leaves one level finer touching B
                    if (c0 < 0) continue;
                    for (int k = 0; k < 4; ++k) {
                        const int ch = c0 + k, cx = t.ix[ch], cy = t.iy[ch];
                        if (!touching(l, ix, iy, l + 1, cx, cy)) continue;
                        const int chl = t.leaf[ch];
                        if (!leaf_ok(t, chl) || chl < 0 || !t.leaf_nz[chl]) continue;
                        const int r = ring_slot(cx - 2 * ix, cy - 2 * iy, -1, 2, 0, 1);
                        if (r >= 0) nr[21 + r] = chl;
                    }
                } else if (l >= 1) {                         // a leaf one level coarser covers (x, y)
                    const int pc = find_box(t, l - 1, x >> 1, y >> 1);
                    if (pc < 0) continue;
                    const int pl = t.leaf[pc];
                    if (!leaf_ok(t, pl) || pl < 0 || !t.leaf_nz[pl]) continue;
                    const int r = ring_slot(ix - 2 * t.ix[pc], iy - 2 * t.iy[pc], -1, 2, 0, 1);
                    if (r >= 0) nr[9 + r] = pl;
                }
            }
    }
    if (l >= 2) {
        const int px = ix >> 1, py = iy >> 1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int c = find_box(t, l - 1, px + dx, py + dy);
                if (c < 0) continue;
                const int cl = t.leaf[c];
                if (!leaf_ok(t, cl)) continue;
                if (cl >= 0) {                               // list i+
                    if ((dx || dy) && t.leaf_nz[cl] && !touching(l, ix, iy, l - 1, px + dx, py + dy)) {
                        const int r = ring_slot(ix - 2 * (px + dx), iy - 2 * (py + dy), -2, 3, -1, 2);
                        if (r >= 0) xl[r] = cl;
                    }
                    continue;
                }
                const int c0 = children_of(t, c);           // list i
                if (c0 < 0) continue;
                for (int k = 0; k < 4; ++k) {
                    const int ch = c0 + k;
                    const int ox = t.ix[ch] - ix, oy = t.iy[ch] - iy;
                    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1) continue;
                    if (!t.box_nz[ch]) continue;
                    const int r = ring_slot(ox, oy, -3, 3, -1, 1);
                    if (r >= 0) vl[r] = ch;
                }
            }
    }
    if (lf >= 0) {                                           // list i-
        int32_t *wl = wlist + (int64_t)lf * kWSlots;
        for (int s = 0; s < kWSlots; ++s) wl[s] = -1;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                const int c = find_box(t, l, ix + dx, iy + dy);
                if (c < 0) continue;
                const int cl = t.leaf[c];
                if (!leaf_ok(t, cl) || cl >= 0) continue;
                const int c0 = children_of(t, c);
                if (c0 < 0) continue;
                for (int k = 0; k < 4; ++k) {
                    const int ch = c0 + k, cx = t.ix[ch], cy = t.iy[ch];
                    if (touching(l, ix, iy, l + 1, cx, cy)) continue;
                    if (!t.box_nz[ch]) continue;
                    const int r = ring_slot(cx - 2 * ix, cy - 2 * iy, -2, 3, -1, 2);
                    if (r >= 0) wl[r] = ch;
                }
            }
    }
}

}  // namespace

// The lists of the plan's tree, built on the device into d.near, d.vlist,
// d.xlist, d.wlist (allocated here) from the boxes already uploaded, then
// copied to the plan's host arrays, which the pass setup reads.  Fails with
// VPX_ERR_STATE if the tree holds an index out of range.
void build_lists_device(vpx_plan *p, cudaStream_t s) {
    DevTree &d = p->dt;
    const int nb = d.n_boxes, nl = d.n_leaves;
    d.near = dev_alloc<int32_t>((size_t)nl * kNearConfigs);
    d.vlist = dev_alloc<int32_t>((size_t)nb * kVSlots);
    d.xlist = dev_alloc<int32_t>((size_t)nb * kXSlots);
    d.wlist = dev_alloc<int32_t>((size_t)nl * kWSlots);
    std::vector<int32_t> ls(p->level_start, p->level_start + d.n_levels + 1);
    int32_t *dls = dev_upload(ls);
    int *status = dev_alloc<int>(1);
    VPX_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    TreeView t{nb, nl, d.n_levels, dls, d.box_morton, d.box_ix, d.box_iy, d.box_child0, d.box_leaf, d.box_nz,
               d.leaf_nz, status};
    for (int l = 0; l < d.n_levels; ++l) {
        const int cnt = p->level_start[l + 1] - p->level_start[l];
        if (cnt <= 0) continue;
        k_lists_level<<<(cnt + 127) / 128, 128, 0, s>>>(t, l, d.near, d.vlist, d.xlist, d.wlist);
        VPX_LAUNCH("k_lists_level");
    }
    p->near.resize((size_t)nl * kNearConfigs);
    p->vlist.resize((size_t)nb * kVSlots);
    p->xlist.resize((size_t)nb * kXSlots);
    p->wlist.resize((size_t)nl * kWSlots);
    int st = 0;
    VPX_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    VPX_CUDA(cudaMemcpyAsync(p->near.data(), d.near, p->near.size() * 4, cudaMemcpyDeviceToHost, s));
    VPX_CUDA(cudaMemcpyAsync(p->vlist.data(), d.vlist, p->vlist.size() * 4, cudaMemcpyDeviceToHost, s));
    VPX_CUDA(cudaMemcpyAsync(p->xlist.data(), d.xlist, p->xlist.size() * 4, cudaMemcpyDeviceToHost, s));
    VPX_CUDA(cudaMemcpyAsync(p->wlist.data(), d.wlist, p->wlist.size() * 4, cudaMemcpyDeviceToHost, s));
    VPX_CUDA(cudaStreamSynchronize(s));
    dev_free(dls);
    dev_free(status);
    if (st != 0) fail(VPX_ERR_STATE, "device list builder: the tree holds an index out of range");
}

}  // namespace vpx
