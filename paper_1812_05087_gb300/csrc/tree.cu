// Quadtree of paper Sec. 3.1 built on the device: Morton keys of the element
// midpoints, LSD radix sort, unique key prefixes per level (empty "zero"
// cells never appear), parent links, the direct-interaction records of the
// leaves and interaction lists (children of the parent's neighbours that are
// not neighbours).  Uniform depth, or adaptive (cells with more than
// leaf_size elements split, leaves at any level); children in Z order
// (left-right, then bottom-top).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include <thread>

#include "internal.h"

namespace {

thread_local long long tl_launches = 0;   // kernel launches of the current build
constexpr int KEY_LEVELS = 16;          // 16 levels -> 32-bit keys
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ uint32_t spread2(uint32_t v) {   // 16 bits -> even bit positions
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__device__ __forceinline__ uint32_t compact2(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}
// Z order: x in the even bits, y in the odd bits, so children run
// bottom-left, bottom-right, top-left, top-right.
__device__ __forceinline__ uint32_t morton(uint32_t ix, uint32_t iy) { return spread2(ix) | (spread2(iy) << 1); }

// ---------------------------------------------------------------- reductions
__global__ void k_bbox(const double *xy, int64_t n, double *part) {
    __shared__ double s[6][256];
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300, lmax = 0.0, bad = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x0 = xy[i], y0 = xy[n + i], x1 = xy[2 * n + i], y1 = xy[3 * n + i];
        double cx = 0.5 * (x0 + x1), cy = 0.5 * (y0 + y1);
        double L = hypot(x1 - x0, y1 - y0);
        if (!(L > 0.0) || !isfinite(cx) || !isfinite(cy)) bad = 1.0;
        mnx = fmin(mnx, cx); mny = fmin(mny, cy); mxx = fmax(mxx, cx); mxy = fmax(mxy, cy);
        lmax = fmax(lmax, L);
    }
    int t = threadIdx.x;
    s[0][t] = mnx; s[1][t] = mny; s[2][t] = -mxx; s[3][t] = -mxy; s[4][t] = -lmax; s[5][t] = -bad;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < 6; ++k) s[k][t] = fmin(s[k][t], s[k][t + w]);
        __syncthreads();
    }
    if (t < 6) part[blockIdx.x * 6 + t] = s[t][0];
}

__global__ void k_keys(const double *xy, int64_t n, double x0, double y0, double w16, uint32_t *key,
                       int32_t *idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double cx = 0.5 * (xy[i] + xy[2 * n + i]), cy = 0.5 * (xy[n + i] + xy[3 * n + i]);
    double fx = floor((cx - x0) / w16), fy = floor((cy - y0) / w16);
    uint32_t ix = (uint32_t)fmin(fmax(fx, 0.0), 65535.0), iy = (uint32_t)fmin(fmax(fy, 0.0), 65535.0);
    key[i] = morton(ix, iy);
    idx[i] = (int32_t)i;
}

// -------------------------------------------------------------------- scans
// exclusive scan of int32 in tiles of SCAN_BLOCK; tile sums to `sums`
__global__ void k_scan_tiles(const int32_t *in, int32_t *out, int64_t n, int32_t *sums) {
    __shared__ int32_t s[SCAN_BLOCK];
    int t = threadIdx.x;
    int64_t i = blockIdx.x * (int64_t)SCAN_BLOCK + t;
    int32_t v = i < n ? in[i] : 0;
    s[t] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        int32_t a = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    if (i < n) out[i] = s[t] - v;
    if (t == SCAN_BLOCK - 1) sums[blockIdx.x] = s[t];
}
__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *offs) {
    int64_t i = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] += offs[blockIdx.x];
}

struct Scratch {      // build-time buffers, freed (stream-ordered) at the end of the build
    std::vector<void *> ptrs;
    cudaStream_t st = nullptr;
    cudaError_t err = cudaSuccess;
    template <class T> T *get(size_t count) {
        void *p = nullptr;
        cudaError_t e = dalloc(&p, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e != cudaSuccess) { err = e; return nullptr; }
        ptrs.push_back(p);
        return (T *)p;
    }
    ~Scratch() { for (void *p : ptrs) dfree(p, st); }
};

// total of an exclusive scan on the device: out[n-1] + in[n-1]
__global__ void k_scan_total(const int32_t *in, const int32_t *out, int64_t n, int32_t *total) {
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0;
}
cudaError_t scan_excl(Scratch &S, cudaStream_t st, const int32_t *in, int32_t *out, int64_t n, int32_t *total);
// exclusive scan whose total stays on the device (no synchronisation)
cudaError_t scan_excl_dev(Scratch &S, cudaStream_t st, const int32_t *in, int32_t *out, int64_t n,
                          int32_t *d_total) {
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb == 0) return cudaMemsetAsync(d_total, 0, sizeof(int32_t), st);
    int32_t *sums = S.get<int32_t>(nb), *soff = S.get<int32_t>(nb);
    if (S.err) return S.err;
    k_scan_tiles<<<nb, SCAN_BLOCK, 0, st>>>(in, out, n, sums); ++tl_launches;
    if (nb > 1) {
        int32_t *dummy = S.get<int32_t>(1);
        if (S.err) return S.err;
        cudaError_t e = scan_excl_dev(S, st, sums, soff, nb, dummy);
        if (e) return e;
        k_scan_add<<<nb, SCAN_BLOCK, 0, st>>>(out, n, soff); ++tl_launches;
    }
    k_scan_total<<<1, 1, 0, st>>>(in, out, n, d_total); ++tl_launches;
    return cudaGetLastError();
}

// exclusive scan, returns the total (synchronises)
cudaError_t scan_excl(Scratch &S, cudaStream_t st, const int32_t *in, int32_t *out, int64_t n,
                      int32_t *total) {
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb == 0) { *total = 0; return cudaSuccess; }
    int32_t *sums = S.get<int32_t>(nb), *soff = S.get<int32_t>(nb);
    if (S.err) return S.err;
    k_scan_tiles<<<nb, SCAN_BLOCK, 0, st>>>(in, out, n, sums); ++tl_launches;
    if (nb > 1) {
        int32_t tot = 0;
        cudaError_t e = scan_excl(S, st, sums, soff, nb, &tot);
        if (e) return e;
        k_scan_add<<<nb, SCAN_BLOCK, 0, st>>>(out, n, soff); ++tl_launches;
        *total = tot;
        return cudaGetLastError();
    }
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, sums, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e) return e;
    e = cudaStreamSynchronize(st);
    *total = h;
    return e;
}

// ------------------------------------------------------------- radix sort
// LSD radix sort of (key, value) pairs, 8 bits per pass, stable.
constexpr int RS_TILE = 256;
__global__ void k_rs_hist(const uint32_t *key, int64_t n, int shift, int32_t *hist, int64_t ntiles) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = blockIdx.x * (int64_t)RS_TILE + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1);
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];   // digit-major
}
__global__ void k_rs_scatter(const uint32_t *key, const int32_t *val, int64_t n, int shift,
                             const int32_t *offs, int64_t ntiles, uint32_t *key2, int32_t *val2) {
    __shared__ int32_t wc[8][256];       // per-warp digit counts
    __shared__ int32_t base[256];
    int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int k = t; k < 8 * 256; k += RS_TILE) (&wc[0][0])[k] = 0;
    __syncthreads();
    int64_t i = blockIdx.x * (int64_t)RS_TILE + t;
    bool ok = i < n;
    uint32_t k = ok ? key[i] : 0u;
    uint32_t d = ok ? ((k >> shift) & 255u) : 256u;
    unsigned mask = __match_any_sync(0xFFFFFFFFu, d);
    int rank = __popc(mask & ((1u << lane) - 1u));
    if (ok && rank == 0) wc[w][d] = __popc(mask);
    __syncthreads();
    // per digit: exclusive prefix over warps (stable: lower warps first)
    {
        int run = 0;
        for (int ww = 0; ww < 8; ++ww) { int c = wc[ww][t]; wc[ww][t] = run; run += c; }
        base[t] = offs[(int64_t)t * ntiles + blockIdx.x];
    }
    __syncthreads();
    if (ok) {
        int64_t pos = base[d] + wc[w][d] + rank;
        key2[pos] = k;
        val2[pos] = val[i];
    }
}

cudaError_t radix_sort(Scratch &S, cudaStream_t st, uint32_t *key, int32_t *val, int64_t n, int bits) {
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    uint32_t *k2 = S.get<uint32_t>(n);
    int32_t *v2 = S.get<int32_t>(n), *hist = S.get<int32_t>(256 * ntiles), *offs = S.get<int32_t>(256 * ntiles);
    int32_t *dtot = S.get<int32_t>(1);         // the scans' totals (n) stay on the device
    if (S.err) return S.err;
    uint32_t *ka = key, *kb = k2;
    int32_t *va = val, *vb = v2;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_TILE, 0, st>>>(ka, n, shift, hist, ntiles); ++tl_launches;
        cudaError_t e = scan_excl_dev(S, st, hist, offs, 256 * ntiles, dtot);
        if (e) return e;
        k_rs_scatter<<<ntiles, RS_TILE, 0, st>>>(ka, va, n, shift, offs, ntiles, kb, vb); ++tl_launches;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != key) {
        cudaMemcpyAsync(key, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(val, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}

// --------------------------------------------------------------- levels
// longest run of equal key prefixes at every level (leaf occupancy)
__global__ void k_runmax(const uint32_t *key, int64_t n, int Lmax, int32_t *runmax) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int L = 0; L <= Lmax; ++L) {
        int sh = 2 * (KEY_LEVELS - L);
        uint32_t p = sh >= 32 ? 0u : (key[i] >> sh);
        if (i > 0 && (sh >= 32 ? 0u : (key[i - 1] >> sh)) == p) continue;
        int64_t lo = i, hi = n;     // first index with a different prefix
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            uint32_t pm = sh >= 32 ? 0u : (key[mid] >> sh);
            if (pm == p) lo = mid; else hi = mid;
        }
        atomicMax(&runmax[L], (int32_t)(hi - i));
    }
}

__global__ void k_flags(const uint32_t *key, int64_t n, int sh, int32_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t p = sh >= 32 ? 0u : key[i] >> sh;
    flag[i] = (i == 0 || (sh >= 32 ? 0u : key[i - 1] >> sh) != p) ? 1 : 0;
}
// cells of one level: start, key, coordinates; element -> cell (level-local)
__global__ void k_cells(const uint32_t *key, int64_t n, int sh, const int32_t *flag, const int32_t *ex,
                        int64_t off, int32_t *cstart, uint32_t *ckey, int32_t *cix, int32_t *ciy,
                        int32_t *elem_cell) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = ex[i] + flag[i] - 1;
    elem_cell[i] = c;
    if (flag[i]) {
        uint32_t p = sh >= 32 ? 0u : key[i] >> sh;
        cstart[off + c] = (int32_t)i;
        ckey[off + c] = p;
        cix[off + c] = (int32_t)compact2(p);
        ciy[off + c] = (int32_t)compact2(p >> 1);
    }
}
__global__ void k_cell_end(const int32_t *cstart, int32_t *cend, int64_t off, int64_t ncell, int64_t n) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    cend[off + c] = (c + 1 < ncell) ? cstart[off + c + 1] : (int32_t)n;
}
__global__ void k_parent(const int32_t *cstart, int64_t off, int64_t ncell, const int32_t *elem_cell_up,
                         int64_t off_up, int32_t *parent) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    parent[off + c] = (int32_t)(off_up + elem_cell_up[cstart[off + c]]);
}

// near-field work items: consecutive target pairs of one leaf (a leaf with an
// odd count ends with a single, second index -1)
__global__ void k_items_count(const int32_t *cstart, const int32_t *cend, const int2 *leaf_at, int64_t nleaf,
                              int32_t *cnt) {
    int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (L >= nleaf) return;
    const int c = leaf_at[L].x;
    cnt[L] = (cend[c] - cstart[c] + 1) / 2;
}
__global__ void k_items_fill(const int32_t *cstart, const int32_t *cend, const int2 *leaf_at, int64_t nleaf,
                             const int32_t *ioff, int2 *items) {
    int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (L >= nleaf) return;
    const int c = leaf_at[L].x;
    const int s0 = cstart[c], s1 = cend[c];
    int o = ioff[L];
    for (int e = s0; e < s1; e += 2) items[o++] = make_int2(e, e + 1 < s1 ? e + 1 : -1);
}

// upward-pass work items: each leaf's elements in chunks of at most cpe
// (leaf, first element, end), so that one block's P2M work is bounded
// whatever the leaf's size
__global__ void k_upitems_count(const int32_t *cstart, const int32_t *cend, const int2 *leaf_at, int64_t nleaf,
                                int cpe, int32_t *cnt) {
    int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (L >= nleaf) return;
    const int c = leaf_at[L].x;
    cnt[L] = (cend[c] - cstart[c] + cpe - 1) / cpe;
}
__global__ void k_upitems_fill(const int32_t *cstart, const int32_t *cend, const int2 *leaf_at, int64_t nleaf,
                               int cpe, const int32_t *ioff, int4 *items) {
    int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (L >= nleaf) return;
    const int c = leaf_at[L].x;
    const int s0 = cstart[c], s1 = cend[c];
    int o = ioff[L];
    for (int e = s0; e < s1; e += cpe) items[o++] = make_int4((int)L, e, min(e + cpe, s1), 0);
}

// the leaves of a uniform tree: every cell of level L
__global__ void k_leaf_uniform(int64_t loff, int64_t nleaf, int L, int2 *leaf_at) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nleaf) leaf_at[i] = make_int2((int)(loff + i), L);
}

__device__ int32_t find_key(const uint32_t *ckey, int64_t off, int64_t ncell, uint32_t k) {
    int64_t lo = 0, hi = ncell;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (ckey[off + mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < ncell && ckey[off + lo] == k) ? (int32_t)lo : -1;
}

// sum of ncell counts (atomic, into one 64-bit total)
__global__ void k_sum_range(const int32_t *cnt, int64_t ncell, unsigned long long *total) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int v = c < ncell ? cnt[c] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, (unsigned long long)v);
}
// direct pairs if the cells of this level were the leaves: own elements x
// elements of the cells sharing a vertex (incl. itself)
__global__ void k_p2p_estimate(const uint32_t *ckey, const int32_t *cix, const int32_t *ciy, const int32_t *cstart,
                               const int32_t *cend, int64_t off, int64_t ncell, int side, unsigned long long *total) {
    // one warp per cell, lane k < 9 looks up neighbour (k / 3 - 1, k % 3 - 1)
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;                   // whole warp
    const int ix = cix[off + c], iy = ciy[off + c];
    long long nb = 0;
    if (lane < 9) {
        const int jx = ix + lane % 3 - 1, jy = iy + lane / 3 - 1;
        if (jx >= 0 && jy >= 0 && jx < side && jy < side) {
            const int32_t j = find_key(ckey, off, ncell, spread2(jx) | (spread2(jy) << 1));
            if (j >= 0) nb = cend[off + j] - cstart[off + j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xFFFFFFFFu, nb, o);
    const unsigned long long v = (unsigned long long)(cend[off + c] - cstart[off + c]) * (unsigned long long)nb;
    if (lane == 0 && v) atomicAdd(total, v);
}

// Direct-interaction records of each leaf P (level lp): pass 0 counts, pass
// 1 fills.  Two leaves interact directly iff their ancestors at the coarser
// of the two levels share a vertex or coincide, so P's sources are
//   (a) the cells of level lp sharing a vertex with P (P included): their
//       whole subtrees, one contiguous element range each (Z order);
//   (b) for each coarser level m < lp, the leaves of level m that share a
//       vertex with P's ancestor at level m.
// Every other pair meets in the M2L of the first level at which its
// ancestors are apart.  In a uniform tree (b) finds nothing (is_leaf null).
// One warp per leaf; lane k < 9 looks up offset (k % 3 - 1, k / 3 - 1), and
// ballots keep the records in that order, level by level.
__global__ void k_recs(const uint32_t *ckey, const int32_t *cix, const int32_t *ciy, const int32_t *cstart,
                       const int32_t *cend, const int32_t *is_leaf, const int64_t *lvoff, const int2 *leaf_at,
                       int64_t nleaf, const int32_t *roff, int4 *tab, int32_t *cnt, int32_t *cmax) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nleaf) return;                   // whole warp
    const int2 P = leaf_at[w];
    const int lp = P.y, ix = cix[P.x], iy = ciy[P.x];
    int m = 0;
    for (int l = lp; l >= 1; --l) {
        if (l < lp && !is_leaf) break;
        const int sh = lp - l, ax = ix >> sh, ay = iy >> sh, side = 1 << l;
        int32_t j = -1;
        if (lane < 9 && (l == lp || lane != 4)) {
            const int jx = ax + lane % 3 - 1, jy = ay + lane / 3 - 1;
            if (jx >= 0 && jy >= 0 && jx < side && jy < side) {
                const int32_t f = find_key(ckey, lvoff[l], lvoff[l + 1] - lvoff[l], morton(jx, jy));
                if (f >= 0 && (l == lp || is_leaf[lvoff[l] + f])) j = (int32_t)(lvoff[l] + f);
            }
        }
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, j >= 0);
        if (tab && j >= 0)
            tab[roff[w] + m + __popc(mask & ((1u << lane) - 1u))] = make_int4(cstart[j], cend[j] - cstart[j], 0, 0);
        m += __popc(mask);
    }
    if (lp == 0) {                            // the root alone: the tree is one leaf
        if (tab && lane == 0) tab[roff[w]] = make_int4(cstart[P.x], cend[P.x] - cstart[P.x], 0, 0);
        m = 1;
    }
    if (cnt && lane == 0) {
        cnt[w] = m;
        atomicMax(cmax, m);
    }
}

// interaction lists of the cells of one level (global cell indices): the
// children of the parent's neighbours that are not neighbours of the cell.
// One warp per cell; candidate k < 36 is child k % 4 of parent neighbour
// (dx, dy) = ((k / 4) % 3 - 1, (k / 4) / 3 - 1), and a ballot keeps the list
// in candidate order.
__global__ void k_ilist(const uint32_t *ckey, const int32_t *cix, const int32_t *ciy, int64_t off,
                        int64_t ncell, int side, const int32_t *iloff, int32_t *ilidx, int32_t *cnt) {
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;                   // whole warp
    const int ix = cix[off + c], iy = ciy[off + c], px = ix >> 1, py = iy >> 1, pside = side >> 1;
    int m = 0;
    for (int base = 0; base < 36; base += 32) {
        const int k = base + lane;
        int32_t j = -1;
        if (k < 36) {
            const int q = k >> 2, ch = k & 3;
            const int qx = px + q % 3 - 1, qy = py + q / 3 - 1;
            if (qx >= 0 && qy >= 0 && qx < pside && qy < pside) {
                const int jx = 2 * qx + (ch & 1), jy = 2 * qy + (ch >> 1);
                if (abs(jx - ix) > 1 || abs(jy - iy) > 1)      // not a neighbour (or itself)
                    j = find_key(ckey, off, ncell, spread2(jx) | (spread2(jy) << 1));
            }
        }
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, j >= 0);
        if (ilidx && j >= 0) ilidx[iloff[off + c] + m + __popc(mask & ((1u << lane) - 1u))] = (int32_t)(off + j);
        m += __popc(mask);
    }
    if (cnt && lane == 0) cnt[off + c] = m;
}

// ------------------------------------------------------------ adaptive tree
// Paper Sec. 3.1: a cell holding more than the prescribed number of elements
// is divided into four children, recursively; otherwise it is a leaf.  The
// cells of every level are first built as for a uniform tree (all non-empty
// key prefixes down to the occupancy depth); the adaptive tree keeps those
// whose every ancestor was split, renumbered in the same (level, key) order.
struct LevelTab {
    const int32_t *ec[KEY_LEVELS + 1];   // sorted element -> its cell of level l (level-local)
    int64_t off[KEY_LEVELS + 2];         // first cell of level l (all non-empty cells)
    int L;                               // deepest level built
};

// deepest level whose cells are at least four times the element's length
// (the rule that bounds how far an element extends past its leaf)
__global__ void k_elem_level(const double *xy, int64_t n, const int32_t *idx, double h0, int32_t *lev) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t e = idx[i];
    const double len = hypot(xy[2 * n + e] - xy[e], xy[3 * n + e] - xy[n + e]);
    const double v = floor(log2(2.0 * h0 / (4.0 * len)) + 1e-12);
    lev[i] = (int32_t)fmin(fmax(v, 0.0), (double)KEY_LEVELS);
}

// minimum element level of every cell: a segmented minimum over each warp's
// run of elements of one cell (cells are runs of consecutive sorted
// elements), then one atomic per run
__global__ void k_cell_minlev(LevelTab T, int64_t n, const int32_t *lev, int32_t *cmin) {
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool ok = i < n;
    const int v0 = ok ? lev[i] : KEY_LEVELS;
    for (int l = 0; l <= T.L; ++l) {
        const int c = ok ? T.ec[l][i] : -1;
        int v = v0;
        for (int o = 1; o < 32; o <<= 1) {
            const int vo = __shfl_down_sync(FULL, v, o), co = __shfl_down_sync(FULL, c, o);
            if (lane + o < 32 && co == c) v = min(v, vo);
        }
        const int cp = __shfl_up_sync(FULL, c, 1);
        if (ok && (lane == 0 || cp != c)) atomicMin(&cmin[T.off[l] + c], v);
    }
}

// a cell of level l is split when it holds more than s elements, l is above
// the deepest level, and every element allows level l + 1; it exists when
// every ancestor is split, and is a leaf when it exists and is not split
__global__ void k_exist(LevelTab T, const int32_t *cstart, const int32_t *cend, const int32_t *parent,
                        const int32_t *cmin, int s, int64_t NC, int32_t *exist, int32_t *leaf) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= NC) return;
    int l = 0;
    while (c >= T.off[l + 1]) ++l;
    auto splits = [&](int64_t a, int la) { return la < T.L && cend[a] - cstart[a] > s && cmin[a] >= la + 1; };
    bool ex = true;
    int64_t a = parent[c];
    for (int la = l - 1; a >= 0; --la) {
        if (!splits(a, la)) {
            ex = false;
            break;
        }
        a = parent[a];
    }
    exist[c] = ex ? 1 : 0;
    leaf[c] = (ex && !splits(c, l)) ? 1 : 0;
}

// the kept cells under their new indices (exclusive scan nidx of exist)
__global__ void k_compact(int64_t NC, const int32_t *exist, const int32_t *nidx, const uint32_t *key,
                          const int32_t *ix, const int32_t *iy, const int32_t *cs, const int32_t *ce,
                          const int32_t *par, const int32_t *leaf, uint32_t *key2, int32_t *ix2, int32_t *iy2,
                          int32_t *cs2, int32_t *ce2, int32_t *par2, int32_t *leaf2) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= NC || !exist[c]) return;
    const int32_t j = nidx[c];
    key2[j] = key[c];
    ix2[j] = ix[c];
    iy2[j] = iy[c];
    cs2[j] = cs[c];
    ce2[j] = ce[c];
    par2[j] = par[c] >= 0 ? nidx[par[c]] : -1;
    leaf2[j] = leaf[c];
}

// per level: first kept cell and first leaf (exclusive scans at the level
// boundaries), levels 0 .. L + 1
__global__ void k_level_counts(LevelTab T, const int32_t *nidx, const int32_t *lidx, int64_t *out) {
    const int l = threadIdx.x;
    if (l > T.L + 1) return;
    out[l] = nidx[T.off[l]];
    out[T.L + 2 + l] = lidx[T.off[l]];
}

// leaves (cell under its new index, level) and each sorted element's leaf
__global__ void k_leaf_table(LevelTab T, int64_t NC, const int32_t *leaf, const int32_t *nidx, const int32_t *lidx,
                             int2 *leaf_at) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= NC || !leaf[c]) return;
    int l = 0;
    while (c >= T.off[l + 1]) ++l;
    leaf_at[lidx[c]] = make_int2(nidx[c], l);
}
__global__ void k_elem_leaf(LevelTab T, int64_t n, const int32_t *leaf, const int32_t *lidx, int32_t *elem_leaf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t r = -1;
    for (int l = 0; l <= T.L && r < 0; ++l) {   // the deepest level's kept cells are leaves
        const int64_t c = T.off[l] + T.ec[l][i];
        if (leaf[c]) r = lidx[c];
    }
    elem_leaf[i] = r;
}

__global__ void k_geom(const double *xy, int64_t n, const int32_t *idx, const int32_t *elem_leaf,
                       const int2 *leaf_at, const int32_t *cix, const int32_t *ciy, double x0, double y0,
                       double h0, double w16, int64_t *perm, float4 *g_rel, float4 *g_frame, float2 *g_grid,
                       float4 *g_loc, double *xys) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t e = idx[i];
    perm[i] = e;
    double ax = xy[e], ay = xy[n + e], bx = xy[2 * n + e], by = xy[3 * n + e];
    xys[i] = ax; xys[n + i] = ay; xys[2 * n + i] = bx; xys[3 * n + i] = by;
    const int2 lf = leaf_at[elem_leaf[i]];
    const double wl = ldexp(2.0 * h0, -lf.y);          // the leaf's width
    double ccx = x0 + (cix[lf.x] + 0.5) * wl, ccy = y0 + (ciy[lf.x] + 0.5) * wl;
    g_rel[i] = make_float4((float)(ax - ccx), (float)(ay - ccy), (float)(bx - ccx), (float)(by - ccy));
    const double gx = fmin(fmax(floor((0.5 * (ax + bx) - x0) / w16), 0.0), 65535.0);
    const double gy = fmin(fmax(floor((0.5 * (ay + by) - y0) / w16), 0.0), 65535.0);
    const double hx = x0 + (gx + 0.5) * w16, hy = y0 + (gy + 0.5) * w16;
    g_grid[i] = make_float2((float)gx, (float)gy);
    g_loc[i] = make_float4((float)(ax - hx), (float)(ay - hy), (float)(bx - hx), (float)(by - hy));
    double L = hypot(bx - ax, by - ay);
    g_frame[i] = make_float4((float)((bx - ax) / L), (float)((by - ay) / L), (float)(0.5 * L), 0.f);
}

// group interaction-list entries by (level, offset)
__global__ void k_mkeys(const int32_t *iloff, const int32_t *ilidx, const int32_t *cix, const int32_t *ciy,
                        const int64_t *lvloff, int L, int64_t first, int64_t ncell, const int32_t *koff,
                        int32_t *kcur, int2 *pairs, int32_t *kcnt) {
    int64_t c = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= first + ncell) return;
    int lvl = 0;
    while (lvl < L && c >= lvloff[lvl + 1]) ++lvl;
    for (int q = iloff[c]; q < iloff[c + 1]; ++q) {
        int32_t J = ilidx[q];
        int key = lvl * 49 + (cix[c] - cix[J] + 3) * 7 + (ciy[c] - ciy[J] + 3);
        if (kcnt) atomicAdd(&kcnt[key], 1);
        else {
            int pos = koff[key] + atomicAdd(&kcur[key], 1);
            pairs[pos] = make_int2((int)c, J);
        }
    }
}

__global__ void k_p2p_count(const int32_t *cstart, const int32_t *cend, const int2 *leaf_at, int64_t nleaf,
                            const int32_t *nboff, const int4 *tab, unsigned long long *tot) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nleaf) return;
    const int lc = leaf_at[c].x;
    long long nt = cend[lc] - cstart[lc], ns = 0;
    for (int k = nboff[c]; k < nboff[c + 1]; ++k) ns += tab[k].y;
    atomicAdd(tot, (unsigned long long)(nt * ns));
}

}  // namespace

#define TRY(call)                                                                   \
    do {                                                                            \
        cudaError_t _e = (call);                                                    \
        if (_e != cudaSuccess) {                                                    \
            tree_free(t);                                                           \
            return ctx_fail(ctx, _e == cudaErrorMemoryAllocation ? DDM_ENOMEM : DDM_ECUDA, \
                            std::string("tree build: ") + #call + ": " + cudaGetErrorString(_e)); \
        }                                                                           \
    } while (0)

// Preconditioner blocks (host): chains of elements sharing end points, cut
// into runs of at most 64 elements; elements on no chain are blocks of one.
struct Chains {
    std::vector<int32_t> boff{0};
    std::vector<int64_t> belem;
    std::vector<int32_t> chain_blk0{0};   // first block of every chain (CSR over chains)
    std::vector<int32_t> pc;              // coarse-level blocks (upload source, lives until the build ends)
};
static void find_chains(const double *hxy, int64_t n, Chains &out) {
    std::vector<int32_t> &boff = out.boff;
    std::vector<int64_t> &belem = out.belem;
    // end points are matched on a grid of 1e-6 of the shortest element
    double lmin = 1e300;
    for (int64_t e = 0; e < n; ++e)
        lmin = std::min(lmin, hypot(hxy[2 * n + e] - hxy[e], hxy[3 * n + e] - hxy[n + e]));
    const double q = 1e-6 * lmin;
    // start points in an open-addressing hash table (quantised coordinates)
    size_t cap = 1;
    while (cap < 2 * (size_t)n) cap <<= 1;
    std::vector<int64_t> slot(cap, -1);
    std::vector<long long> skx(cap), sky(cap);
    auto hidx = [&](long long kx, long long ky) {
        uint64_t h = (uint64_t)kx * 0x9E3779B97F4A7C15ull ^ ((uint64_t)ky + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
        return (size_t)((h ^ (h >> 29)) & (cap - 1));
    };
    auto qz = [&](double v) { return (long long)llround(v / q); };
    for (int64_t e = 0; e < n; ++e) {      // a repeated start point keeps the last element
        long long kx = qz(hxy[e]), ky = qz(hxy[n + e]);
        size_t i = hidx(kx, ky);
        while (slot[i] >= 0 && !(skx[i] == kx && sky[i] == ky)) i = (i + 1) & (cap - 1);
        slot[i] = e;
        skx[i] = kx;
        sky[i] = ky;
    }
    std::vector<int64_t> next(n, -1), prevc(n, 0);
    for (int64_t e = 0; e < n; ++e) {
        long long kx = qz(hxy[2 * n + e]), ky = qz(hxy[3 * n + e]);
        size_t i = hidx(kx, ky);
        while (slot[i] >= 0 && !(skx[i] == kx && sky[i] == ky)) i = (i + 1) & (cap - 1);
        int64_t f = slot[i];
        if (f >= 0 && f != e && prevc[f] == 0) {
            next[e] = f;
            prevc[f] = 1;
        }
    }
    std::vector<char> seen(n, 0);
    const int BMAX = 64;
    auto emit_chain = [&](int64_t head) {
        int cnt = 0;
        for (int64_t e = head; e >= 0 && !seen[e]; e = next[e]) {
            seen[e] = 1;
            belem.push_back(e);
            if (++cnt == BMAX) {
                boff.push_back((int32_t)belem.size());
                cnt = 0;
            }
        }
        if (cnt) boff.push_back((int32_t)belem.size());
        out.chain_blk0.push_back((int32_t)boff.size() - 1);
    };
    for (int64_t e = 0; e < n; ++e)
        if (!prevc[e]) emit_chain(e);
    for (int64_t e = 0; e < n; ++e)          // closed loops
        if (!seen[e]) emit_chain(e);
}

void tree_free(ddm_tree *t) {
    if (!t) return;
    void *ps[] = {t->mk_work, t->pb_off, t->pb_elem, t->pb_moff, t->pb_inv, t->pc_blk, t->pc_inv, t->mk_off, t->mk_pair, t->perm, t->cell_key, t->cell_ix, t->cell_iy, t->cell_start, t->cell_end, t->cell_parent,
                  t->il_off, t->il_idx, t->nb_off, t->leaf_at, t->nb_tab, t->near_items, t->up_items, t->elem_leaf, t->g_rel, t->g_frame, t->g_grid, t->g_loc,
                  t->xy_sorted, t->xy_caller, t->W, t->Fl, t->far4, t->chg, t->lv_off, t->lv_pair, t->lv_work,
                  t->Wc, t->Gc};
    for (void *p : ps) dfree(p, t->stream);
    for (double *p : t->win_blk) dfree(p, t->stream);
    for (float *p : t->ops_set) dfree(p, t->stream);
    for (float *p : t->svd_set) dfree(p, t->stream);
    delete t;
}

static ddm_status tree_build_one(ddm_ctx *ctx, const double *d_xy, int64_t n, const ddm_fmm_params &prm,
                                 ddm_tree **out) {
    if (!ctx || !d_xy || !out || n <= 0 || n > (int64_t)1 << 30)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_build_tree: bad arguments");
    cudaStream_t st = ctx->stream;
    ddm_tree *t = new ddm_tree();
    t->n = n;
    t->prm = prm;
    Scratch S;
    S.st = st;
    t->stream = st;
    tl_launches = 0;
    prof_begin(ctx, 9);
    const int TB = 256;
    int64_t nbk = (n + TB - 1) / TB;

    // bounding square of the midpoints
    int nbb = (int)std::min<int64_t>(nbk, 1024);
    double *part = S.get<double>(6 * nbb);
    TRY(S.err);
    k_bbox<<<nbb, 256, 0, st>>>(d_xy, n, part); ++tl_launches;
    std::vector<double> hp(6 * nbb);
    TRY(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300, lmax = 0, bad = 0;
    for (int b = 0; b < nbb; ++b) {
        mnx = std::min(mnx, hp[6 * b]); mny = std::min(mny, hp[6 * b + 1]);
        mxx = std::max(mxx, -hp[6 * b + 2]); mxy = std::max(mxy, -hp[6 * b + 3]);
        lmax = std::max(lmax, -hp[6 * b + 4]); bad = std::max(bad, -hp[6 * b + 5]);
    }
    if (bad > 0) { tree_free(t); return ctx_fail(ctx, DDM_EINVAL, "ddm_build_tree: zero-length or non-finite element"); }
    // end points to the host (context's pinned buffer) for the chain search,
    // which runs on a worker thread while the device builds the tree
    if (ctx->h_pin_cap < 4 * n) {
        if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
        ctx->h_pin = nullptr;
        ctx->h_pin_cap = 0;
        TRY(cudaMallocHost(&ctx->h_pin, 4 * n * sizeof(double)));
        ctx->h_pin_cap = 4 * n;
    }
    cudaEvent_t xy_ev;
    TRY(cudaEventCreateWithFlags(&xy_ev, cudaEventDisableTiming));
    TRY(cudaMemcpyAsync(ctx->h_pin, d_xy, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(cudaEventRecord(xy_ev, st));
    Chains chains;
    bool chain_ok = true;
    const double *hxy_pin = ctx->h_pin;
    std::thread chain_th([&chains, &chain_ok, xy_ev, hxy_pin, n]() {
        if (cudaEventSynchronize(xy_ev) != cudaSuccess) { chain_ok = false; return; }
        find_chains(hxy_pin, n, chains);
    });
    bool chain_th_live = true;
    // a failing step below must not leave the worker running
    struct Joiner {
        std::thread &th;
        bool &live;
        cudaEvent_t ev;
        ~Joiner() {
            if (live && th.joinable()) th.join();
            cudaEventDestroy(ev);
        }
    } joiner{chain_th, chain_th_live, xy_ev};
    double span = std::max(std::max(mxx - mnx, mxy - mny), 4.0 * lmax);
    double h0 = 0.5 * span * (1.0 + 1e-9) + 1e-300;
    t->cx = 0.5 * (mnx + mxx); t->cy = 0.5 * (mny + mxy); t->h0 = h0;
    double X0 = t->cx - h0, Y0 = t->cy - h0;

    // keys at 16 levels, sort
    uint32_t *key = S.get<uint32_t>(n);
    int32_t *idx = S.get<int32_t>(n);
    TRY(S.err);
    double w16 = 2.0 * h0 / 65536.0;
    k_keys<<<nbk, TB, 0, st>>>(d_xy, n, X0, Y0, w16, key, idx); ++tl_launches;
    TRY(radix_sort(S, st, key, idx, n, 32));

    // depth: smallest L whose leaves hold <= leaf_size, capped so that the
    // longest element is at most a quarter of a leaf (adaptive: the cap is
    // applied per cell, below)
    int Lcap = prm.adaptive ? KEY_LEVELS : (int)std::floor(std::log2(2.0 * h0 / (4.0 * lmax)) + 1e-12);
    Lcap = std::max(0, std::min(Lcap, KEY_LEVELS));
    if (prm.max_depth > 0) Lcap = std::min(Lcap, prm.max_depth);
    int32_t *runmax = S.get<int32_t>(KEY_LEVELS + 1);
    TRY(S.err);
    TRY(cudaMemsetAsync(runmax, 0, (KEY_LEVELS + 1) * sizeof(int32_t), st));
    k_runmax<<<nbk, TB, 0, st>>>(key, n, Lcap, runmax); ++tl_launches;
    int32_t hrun[KEY_LEVELS + 1];
    TRY(cudaMemcpyAsync(hrun, runmax, sizeof(hrun), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    int L = Lcap;
    for (int l = 0; l <= Lcap; ++l)
        if (hrun[l] <= prm.leaf_size) { L = l; break; }
    t->depth = L;
    t->adaptive = prm.adaptive;

    // cells of every level
    std::vector<int32_t *> ecell(L + 1);
    int32_t *flag = S.get<int32_t>(n), *ex = S.get<int32_t>(n);
    TRY(S.err);
    std::vector<int64_t> ncl(L + 1);
    t->lvl_off.assign(L + 2, 0);
    int32_t *d_ncl = S.get<int32_t>(L + 1);
    TRY(S.err);
    for (int l = 0; l <= L; ++l) {       // cell counts of all levels, read back once
        k_flags<<<nbk, TB, 0, st>>>(key, n, 2 * (KEY_LEVELS - l), flag); ++tl_launches;
        TRY(scan_excl_dev(S, st, flag, ex, n, d_ncl + l));
        ecell[l] = S.get<int32_t>(n);
        TRY(S.err);
        TRY(cudaMemcpyAsync(ecell[l], ex, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        // stash flags in ecell temporarily: ecell = ex + flag - 1 computed in k_cells later
        int32_t *fl = S.get<int32_t>(n);
        TRY(S.err);
        TRY(cudaMemcpyAsync(fl, flag, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        ecell.push_back(fl);   // keep alive; index L+1+l
    }
    {
        std::vector<int32_t> h(L + 1);
        TRY(cudaMemcpyAsync(h.data(), d_ncl, (L + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        for (int l = 0; l <= L; ++l) {
            ncl[l] = h[l];
            t->lvl_off[l + 1] = t->lvl_off[l] + h[l];
        }
    }
    int64_t NC = t->lvl_off[L + 1];
    t->n_cells = NC;
    TRY(dalloc(&t->cell_key, NC * sizeof(uint32_t), st));
    TRY(dalloc(&t->cell_ix, NC * sizeof(int32_t), st));
    TRY(dalloc(&t->cell_iy, NC * sizeof(int32_t), st));
    TRY(dalloc(&t->cell_start, NC * sizeof(int32_t), st));
    TRY(dalloc(&t->cell_end, NC * sizeof(int32_t), st));
    TRY(dalloc(&t->cell_parent, NC * sizeof(int32_t), st));
    for (int l = 0; l <= L; ++l) {
        int32_t *fl = ecell[L + 1 + l];
        int32_t *exl = ecell[l];
        int32_t *elem_cell = S.get<int32_t>(n);
        TRY(S.err);
        k_cells<<<nbk, TB, 0, st>>>(key, n, 2 * (KEY_LEVELS - l), fl, exl, t->lvl_off[l], t->cell_start,
                                   t->cell_key, t->cell_ix, t->cell_iy, elem_cell); ++tl_launches;
        ecell[l] = elem_cell;
        int64_t nc = ncl[l];
        k_cell_end<<<(nc + TB - 1) / TB, TB, 0, st>>>(t->cell_start, t->cell_end, t->lvl_off[l], nc, n); ++tl_launches;
    }
    TRY(cudaMemsetAsync(t->cell_parent, 0xFF, sizeof(int32_t), st));   // root: -1
    for (int l = 1; l <= L; ++l) {
        int64_t nc = ncl[l];
        k_parent<<<(nc + TB - 1) / TB, TB, 0, st>>>(t->cell_start, t->lvl_off[l], nc, ecell[l - 1],
                                                   t->lvl_off[l - 1], t->cell_parent); ++tl_launches;
    }

    // depth by cost model: the occupancy rule gives the deepest useful
    // depth; shallower depths trade M2L and tree passes for more direct
    // pairs.  Costs per unit measured on GB300 for n = 8 (near pair 19.4 ps,
    // interaction pair 3.5 ns scaling with n^4, cell 25 ns).
    int32_t *il_cnt = nullptr;                 // interaction-list counts of the depth choice, kept
    int32_t *a_leaf = nullptr, *a_lidx = nullptr;   // adaptive: leaf flags and leaf numbering (all cells)
    int32_t *is_leaf = nullptr;                      // adaptive: leaf flags of the kept cells
    LevelTab LT{};
    if (prm.adaptive) {
        // keep the cells whose ancestors are all split (k_exist), renumbered
        for (int l = 0; l <= L; ++l) {
            LT.ec[l] = ecell[l];
            LT.off[l] = t->lvl_off[l];
        }
        LT.off[L + 1] = NC;
        LT.L = L;
        int32_t *lev = S.get<int32_t>(n), *cmin = S.get<int32_t>(NC), *ex = S.get<int32_t>(NC + 1);
        int32_t *nidx = S.get<int32_t>(NC + 1);
        a_leaf = S.get<int32_t>(NC + 1);
        a_lidx = S.get<int32_t>(NC + 1);
        int64_t *lc = S.get<int64_t>(2 * (L + 2));
        TRY(S.err);
        k_elem_level<<<nbk, TB, 0, st>>>(d_xy, n, idx, h0, lev); ++tl_launches;
        TRY(cudaMemsetAsync(cmin, 0x7F, NC * sizeof(int32_t), st));
        k_cell_minlev<<<nbk, TB, 0, st>>>(LT, n, lev, cmin); ++tl_launches;
        const int64_t cb = (NC + TB - 1) / TB;
        k_exist<<<cb, TB, 0, st>>>(LT, t->cell_start, t->cell_end, t->cell_parent, cmin, prm.leaf_size, NC, ex,
                                   a_leaf); ++tl_launches;
        TRY(scan_excl_dev(S, st, ex, nidx, NC, nidx + NC));
        TRY(scan_excl_dev(S, st, a_leaf, a_lidx, NC, a_lidx + NC));
        k_level_counts<<<1, 32, 0, st>>>(LT, nidx, a_lidx, lc); ++tl_launches;
        std::vector<int64_t> hl(2 * (L + 2));
        TRY(cudaMemcpyAsync(hl.data(), lc, hl.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        const int64_t NCa = hl[L + 1];
        int La = 0;                               // deepest level with a kept cell
        for (int l = 0; l <= L; ++l)
            if (hl[l + 1] > hl[l]) La = l;
        t->leaf_level_min = -1;
        for (int l = 0; l <= L && t->leaf_level_min < 0; ++l)
            if (hl[L + 2 + l + 1] > hl[L + 2 + l]) t->leaf_level_min = l;
        t->n_leaf = hl[L + 2 + L + 1];
        is_leaf = S.get<int32_t>(NCa + 1);
        TRY(S.err);
        uint32_t *key2 = nullptr;
        int32_t *a2[5] = {};                      // ix, iy, start, end, parent of the kept cells
        cudaError_t ae = dalloc(&key2, NCa * sizeof(uint32_t), st);
        for (int k = 0; k < 5 && ae == cudaSuccess; ++k) ae = dalloc(&a2[k], NCa * sizeof(int32_t), st);
        if (ae != cudaSuccess) {
            dfree(key2, st);
            for (int32_t *p : a2) dfree(p, st);
            TRY(ae);
        }
        k_compact<<<cb, TB, 0, st>>>(NC, ex, nidx, t->cell_key, t->cell_ix, t->cell_iy, t->cell_start, t->cell_end,
                                     t->cell_parent, a_leaf, key2, a2[0], a2[1], a2[2], a2[3], a2[4], is_leaf);
        ++tl_launches;
        dfree(t->cell_key, st);
        dfree(t->cell_ix, st);
        dfree(t->cell_iy, st);
        dfree(t->cell_start, st);
        dfree(t->cell_end, st);
        dfree(t->cell_parent, st);
        t->cell_key = key2;
        t->cell_ix = a2[0];
        t->cell_iy = a2[1];
        t->cell_start = a2[2];
        t->cell_end = a2[3];
        t->cell_parent = a2[4];
        TRY(dalloc(&t->leaf_at, std::max<int64_t>(t->n_leaf, 1) * sizeof(int2), st));
        k_leaf_table<<<cb, TB, 0, st>>>(LT, NC, a_leaf, nidx, a_lidx, t->leaf_at); ++tl_launches;
        // (the element -> leaf map, from a_leaf and a_lidx, is written with the geometry below)
        // the kept tree: its levels, cell counts and leaf flags (compact numbering)
        L = La;
        t->depth = L;
        t->lvl_off.assign(L + 2, 0);
        ncl.assign(L + 1, 0);
        for (int l = 0; l <= L; ++l) {
            t->lvl_off[l + 1] = hl[l + 1];
            ncl[l] = hl[l + 1] - hl[l];
        }
        NC = NCa;
        t->n_cells = NC;
    } else if (L >= 3 && prm.max_depth == 0) {
        const int L0 = std::max(2, L - 4), NCAND = L - L0 + 1;
        int32_t *ccnt = S.get<int32_t>(NC + 1);
        il_cnt = ccnt;
        unsigned long long *dsum = S.get<unsigned long long>(2 * (L + 1));   // M2L pairs per level, near pairs per depth
        TRY(S.err);
        TRY(cudaMemsetAsync(dsum, 0, 2 * (L + 1) * sizeof(unsigned long long), st));
        TRY(cudaMemsetAsync(ccnt, 0, (NC + 1) * sizeof(int32_t), st));
        for (int l = 2; l <= L; ++l) {
            int64_t nc = ncl[l];
            k_ilist<<<(32 * nc + TB - 1) / TB, TB, 0, st>>>(t->cell_key, t->cell_ix, t->cell_iy, t->lvl_off[l], nc,
                                                           1 << l, nullptr, nullptr, ccnt); ++tl_launches;
            k_sum_range<<<(nc + TB - 1) / TB, TB, 0, st>>>(ccnt, nc, dsum + l); ++tl_launches;
        }
        for (int Lc = L0; Lc <= L; ++Lc) {
            int64_t nc = ncl[Lc];
            k_p2p_estimate<<<(32 * nc + TB - 1) / TB, TB, 0, st>>>(t->cell_key, t->cell_ix, t->cell_iy, t->cell_start,
                                                             t->cell_end, t->lvl_off[Lc], nc, 1 << Lc,
                                                             dsum + (L + 1) + Lc); ++tl_launches;
        }
        std::vector<unsigned long long> hs(2 * (L + 1));
        TRY(cudaMemcpyAsync(hs.data(), dsum, hs.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        double nfac = std::pow(prm.n_cheb / 8.0, 4.0);
        double best = 1e300;
        int bestL = L;
        (void)NCAND;
        for (int Lc = L0; Lc <= L; ++Lc) {
            long long m2l = 0, cells = 0;
            for (int l = 2; l <= Lc; ++l) m2l += (long long)hs[l];
            for (int l = 0; l <= Lc; ++l) cells += ncl[l];
            double cost = 21.5e-12 * (double)hs[L + 1 + Lc] + 3.5e-9 * nfac * (double)m2l + 25e-9 * (double)cells;
            if (cost < best) { best = cost; bestL = Lc; }
        }
        L = bestL;
        t->depth = L;
        t->lvl_off.resize(L + 2);
        NC = t->lvl_off[L + 1];      // cells of the levels kept
        t->n_cells = NC;
    }

    // leaves (a uniform tree: the cells of level L)
    int64_t *lvd = S.get<int64_t>(L + 2);     // level offsets on the device
    TRY(S.err);
    TRY(cudaMemcpyAsync(lvd, t->lvl_off.data(), (L + 2) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (!prm.adaptive) {
        t->n_leaf = ncl[L];
        t->leaf_level_min = L;
        TRY(dalloc(&t->leaf_at, std::max<int64_t>(t->n_leaf, 1) * sizeof(int2), st));
        k_leaf_uniform<<<(unsigned)std::max<int64_t>((t->n_leaf + TB - 1) / TB, 1), TB, 0, st>>>(
            t->lvl_off[L], t->n_leaf, L, t->leaf_at); ++tl_launches;
    }
    const int64_t nleaf = t->n_leaf;
    int32_t *cnt = S.get<int32_t>(std::max<int64_t>(NC, nleaf) + 1);
    TRY(S.err);
    TRY(dalloc(&t->nb_off, (nleaf + 1) * sizeof(int32_t), st));
    int64_t lb = (nleaf + TB - 1) / TB;
    const int64_t lbw = (32 * nleaf + TB - 1) / TB;   // one warp per leaf
    // direct-interaction records: counts, offsets, records (list sizes are
    // bounded from above, so that the totals can stay on the device until
    // the one read-back below: 9 same-level cells, 8 leaves per coarser level)
    int32_t *rmax = S.get<int32_t>(1);
    TRY(S.err);
    TRY(cudaMemsetAsync(rmax, 0, sizeof(int32_t), st));
    k_recs<<<lbw, TB, 0, st>>>(t->cell_key, t->cell_ix, t->cell_iy, t->cell_start, t->cell_end, is_leaf, lvd,
                               t->leaf_at, nleaf, nullptr, nullptr, cnt, rmax); ++tl_launches;
    TRY(scan_excl_dev(S, st, cnt, t->nb_off, nleaf, t->nb_off + nleaf));
    const int64_t nb_cap = std::max<int64_t>((9 + (is_leaf ? 8 * std::max(L - 1, 0) : 0)) * nleaf, 1);
    TRY(dalloc(&t->nb_tab, nb_cap * sizeof(int4), st));
    k_recs<<<lbw, TB, 0, st>>>(t->cell_key, t->cell_ix, t->cell_iy, t->cell_start, t->cell_end, is_leaf, lvd,
                               t->leaf_at, nleaf, t->nb_off, t->nb_tab, nullptr, nullptr); ++tl_launches;
    const int32_t *d_itot = nullptr;
    {   // near-field work items (target pairs per leaf)
        int32_t *icnt = S.get<int32_t>(nleaf + 1), *ioff = S.get<int32_t>(nleaf + 1);
        TRY(S.err);
        k_items_count<<<lb, TB, 0, st>>>(t->cell_start, t->cell_end, t->leaf_at, nleaf, icnt); ++tl_launches;
        TRY(scan_excl_dev(S, st, icnt, ioff, nleaf, ioff + nleaf));
        TRY(dalloc(&t->near_items, std::max<int64_t>(n, 1) * sizeof(int2), st));   // <= one item per element
        k_items_fill<<<lb, TB, 0, st>>>(t->cell_start, t->cell_end, t->leaf_at, nleaf, ioff, t->near_items);
        ++tl_launches;
        d_itot = ioff + nleaf;
    }
    const int32_t *d_utot = nullptr;
    {   // upward-pass items: about 1024 Gauss points (n per element) per block
        const int cpe = std::max(1, 1024 / prm.n_cheb);
        int32_t *ucnt = S.get<int32_t>(nleaf + 1), *uoff = S.get<int32_t>(nleaf + 1);
        TRY(S.err);
        k_upitems_count<<<lb, TB, 0, st>>>(t->cell_start, t->cell_end, t->leaf_at, nleaf, cpe, ucnt); ++tl_launches;
        TRY(scan_excl_dev(S, st, ucnt, uoff, nleaf, uoff + nleaf));
        // <= one item per leaf plus one per cpe elements
        TRY(dalloc(&t->up_items, (nleaf + n / cpe + 1) * sizeof(int4), st));
        k_upitems_fill<<<lb, TB, 0, st>>>(t->cell_start, t->cell_end, t->leaf_at, nleaf, cpe, uoff, t->up_items);
        ++tl_launches;
        d_utot = uoff + nleaf;
    }

    // interaction lists, levels >= 2: the counts (the depth choice already
    // counted every level it kept; the cells of those levels keep their
    // indices), then the lists
    if (il_cnt) {
        TRY(cudaMemcpyAsync(cnt, il_cnt, NC * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    } else {
        TRY(cudaMemsetAsync(cnt, 0, NC * sizeof(int32_t), st));
        for (int l = 2; l <= L; ++l) {
            int64_t nc = ncl[l];
            k_ilist<<<(32 * nc + TB - 1) / TB, TB, 0, st>>>(t->cell_key, t->cell_ix, t->cell_iy, t->lvl_off[l], nc,
                                                           1 << l, nullptr, nullptr, cnt); ++tl_launches;
        }
    }
    TRY(dalloc(&t->il_off, (NC + 1) * sizeof(int32_t), st));
    TRY(scan_excl_dev(S, st, cnt, t->il_off, NC, t->il_off + NC));
    // <= 27 entries per cell of levels >= 2
    const int64_t il_cap = std::max<int64_t>(27 * (NC - (L >= 2 ? t->lvl_off[2] : NC)), 1);
    TRY(dalloc(&t->il_idx, il_cap * sizeof(int32_t), st));
    for (int l = 2; l <= L; ++l) {
        int64_t nc = ncl[l];
        k_ilist<<<(32 * nc + TB - 1) / TB, TB, 0, st>>>(t->cell_key, t->cell_ix, t->cell_iy, t->lvl_off[l], nc,
                                                       1 << l, t->il_off, t->il_idx, nullptr); ++tl_launches;
    }
    // host sources of uploads, alive until the synchronisation that ends the build
    std::vector<int2> work;
    std::vector<int64_t> moff;
    // M2L pairs grouped by (level, offset)
    {
        int nk = (L + 1) * 49;
        t->n_keys = nk;
        int32_t *kc = S.get<int32_t>(nk + 1), *kcur = S.get<int32_t>(nk);
        const int64_t *lo = lvd;
        TRY(S.err);
        TRY(cudaMemsetAsync(kc, 0, (nk + 1) * sizeof(int32_t), st));
        TRY(cudaMemsetAsync(kcur, 0, nk * sizeof(int32_t), st));
        TRY(dalloc(&t->mk_off, (nk + 1) * sizeof(int32_t), st));
        TRY(dalloc(&t->mk_pair, il_cap * sizeof(int2), st));
        int64_t first = L >= 2 ? t->lvl_off[2] : NC, ncm = NC - first;
        if (ncm > 0) {
            k_mkeys<<<(ncm + 255) / 256, 256, 0, st>>>(t->il_off, t->il_idx, t->cell_ix, t->cell_iy, lo, L, first, ncm,
                                                       nullptr, nullptr, nullptr, kc); ++tl_launches;
        }
        TRY(scan_excl_dev(S, st, kc, t->mk_off, nk, t->mk_off + nk));
        if (ncm > 0) {
            k_mkeys<<<(ncm + 255) / 256, 256, 0, st>>>(t->il_off, t->il_idx, t->cell_ix, t->cell_iy, lo, L, first, ncm,
                                                       t->mk_off, kcur, t->mk_pair, nullptr); ++tl_launches;
        }
        t->ops_n = 0;
        t->ops_cap = 0;
        t->win_clock = 0;
        // one read-back: the group offsets, the near-field item count and the
        // interaction-list total
        int32_t *hdev = S.get<int32_t>(nk + 5);
        TRY(S.err);
        TRY(cudaMemcpyAsync(hdev, t->mk_off, (nk + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        TRY(cudaMemcpyAsync(hdev + nk + 1, d_itot, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        TRY(cudaMemcpyAsync(hdev + nk + 2, t->il_off + NC, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        TRY(cudaMemcpyAsync(hdev + nk + 3, rmax, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        TRY(cudaMemcpyAsync(hdev + nk + 4, d_utot, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        std::vector<int32_t> hk(nk + 5);
        TRY(cudaMemcpyAsync(hk.data(), hdev, (nk + 5) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        t->n_items = hk[nk + 1];
        t->n_m2l = hk[nk + 2];
        t->max_recs = hk[nk + 3];
        t->n_up_items = hk[nk + 4];
        t->max_group = 0;
        for (int k = 0; k < nk; ++k) {
            t->max_group = std::max(t->max_group, hk[k + 1] - hk[k]);
            for (int p0 = hk[k]; p0 < hk[k + 1]; p0 += 64) work.push_back(make_int2(k, p0));
        }
        t->n_work = (int)work.size();
        TRY(dalloc(&t->mk_work, std::max<size_t>(work.size(), 1) * sizeof(int2), st));
        if (!work.empty())
            TRY(cudaMemcpyAsync(t->mk_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    }

    // sorted geometry
    TRY(dalloc(&t->perm, n * sizeof(int64_t), st));
    TRY(dalloc(&t->elem_leaf, n * sizeof(int32_t), st));
    TRY(dalloc(&t->g_rel, n * sizeof(float4), st));
    TRY(dalloc(&t->g_frame, n * sizeof(float4), st));
    TRY(dalloc(&t->g_grid, n * sizeof(float2), st));
    TRY(dalloc(&t->g_loc, n * sizeof(float4), st));
    TRY(dalloc(&t->xy_sorted, 4 * n * sizeof(double), st));
    TRY(dalloc(&t->xy_caller, 4 * n * sizeof(double), st));
    TRY(cudaMemcpyAsync(t->xy_caller, d_xy, 4 * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TRY(dalloc(&t->chg, n * sizeof(float4), st));
    if (prm.adaptive) {
        k_elem_leaf<<<nbk, TB, 0, st>>>(LT, n, a_leaf, a_lidx, t->elem_leaf); ++tl_launches;
    } else {                                  // level-local cell index of level L = leaf index
        TRY(cudaMemcpyAsync(t->elem_leaf, ecell[L], n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    }
    k_geom<<<nbk, TB, 0, st>>>(d_xy, n, idx, t->elem_leaf, t->leaf_at, t->cell_ix, t->cell_iy, X0, Y0, h0, w16,
                              t->perm, t->g_rel, t->g_frame, t->g_grid, t->g_loc, t->xy_sorted); ++tl_launches;
    t->g16 = (float)w16;
    // preconditioner blocks: the chain search (host worker thread, started
    // after the bounding box) is joined here
    {
        chain_th.join();
        chain_th_live = false;
        if (!chain_ok) { tree_free(t); return ctx_fail(ctx, DDM_ECUDA, "tree build: end point copy failed"); }
        std::vector<int32_t> &boff = chains.boff;
        std::vector<int64_t> &belem = chains.belem;
        moff.assign(1, 0);
        t->n_pblk = (int64_t)boff.size() - 1;
        t->pb_max = 0;
        for (int64_t b = 0; b < t->n_pblk; ++b) {
            int m = boff[b + 1] - boff[b];
            t->pb_max = std::max(t->pb_max, m);
            moff.push_back(moff.back() + (int64_t)9 * m * m);
        }
        t->pb_msize = moff.back();
        TRY(dalloc(&t->pb_off, boff.size() * sizeof(int32_t), st));
        TRY(dalloc(&t->pb_elem, std::max<size_t>(belem.size(), 1) * sizeof(int64_t), st));
        TRY(dalloc(&t->pb_moff, moff.size() * sizeof(int64_t), st));
        TRY(cudaMemcpyAsync(t->pb_off, boff.data(), boff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->pb_elem, belem.data(), belem.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->pb_moff, moff.data(), moff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        t->pb_inv = nullptr;
        t->pb_dt = -1.0;
        t->pb_sys = -1;
        // coarse level: the blocks of every chain of at least PC_MIN_BLOCKS blocks
        std::vector<int32_t> &pc = chains.pc;
        for (size_t c = 0; c + 1 < chains.chain_blk0.size(); ++c)
            if (chains.chain_blk0[c + 1] - chains.chain_blk0[c] >= PC_MIN_BLOCKS)
                for (int32_t b = chains.chain_blk0[c]; b < chains.chain_blk0[c + 1]; ++b) pc.push_back(b);
        t->n_pc = (int64_t)pc.size();
        t->pc_modes = 0;
        for (int k = PC_MODES; k >= 1 && !t->pc_modes; --k)
            if (t->n_pc * 3 * k <= PC_MAX_DIM) t->pc_modes = k;
        if (!t->pc_modes) t->n_pc = 0;
        t->pc_blk = nullptr;
        t->pc_inv = nullptr;
        if (t->n_pc) {
            TRY(dalloc(&t->pc_blk, pc.size() * sizeof(int32_t), st));
            TRY(cudaMemcpyAsync(t->pc_blk, pc.data(), pc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        }
    }
    unsigned long long *ptot = S.get<unsigned long long>(1);
    TRY(S.err);
    TRY(cudaMemsetAsync(ptot, 0, sizeof(unsigned long long), st));
    k_p2p_count<<<lb, TB, 0, st>>>(t->cell_start, t->cell_end, t->leaf_at, nleaf, t->nb_off, t->nb_tab, ptot);
    ++tl_launches;
    unsigned long long hp2p = 0;
    TRY(cudaMemcpyAsync(&hp2p, ptot, sizeof(hp2p), cudaMemcpyDeviceToHost, st));
    TRY(cudaGetLastError());
    TRY(cudaStreamSynchronize(st));
    t->n_p2p = (int64_t)hp2p;
    prof_end(ctx, 9, (int)tl_launches);
    *out = t;
    return DDM_OK;
}

// The measured cost model of one product that also picks the uniform tree's
// depth: near pairs, interaction pairs (scaling with n^4) and cells.
static double product_cost_model(const ddm_tree *t) {
    return 21.5e-12 * (double)t->n_p2p + 3.5e-9 * std::pow(t->prm.n_cheb / 8.0, 4.0) * (double)t->n_m2l +
           25e-9 * (double)t->n_cells;
}

// adaptive = 2: both trees, the one the cost model prefers is kept
ddm_status tree_build(ddm_ctx *ctx, const double *d_xy, int64_t n, const ddm_fmm_params &prm, ddm_tree **out) {
    if (prm.adaptive != 2) return tree_build_one(ctx, d_xy, n, prm, out);
    if (!out) return ctx_fail(ctx, DDM_EINVAL, "ddm_build_tree: bad arguments");
    ddm_fmm_params pu = prm, pa = prm;
    pu.adaptive = 0;
    pa.adaptive = 1;
    ddm_tree *tu = nullptr, *ta = nullptr;
    ddm_status st = tree_build_one(ctx, d_xy, n, pu, &tu);
    if (st) return st;
    if ((st = tree_build_one(ctx, d_xy, n, pa, &ta))) {
        tree_free(tu);
        return st;
    }
    const bool pick_a = product_cost_model(ta) < product_cost_model(tu);
    tree_free(pick_a ? tu : ta);
    *out = pick_a ? ta : tu;
    return DDM_OK;
}
