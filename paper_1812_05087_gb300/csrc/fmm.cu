// Influence products of paper Eqs. (2.3)-(2.5) on the GPU.
//
//  FMM path (paper Sec. 3, black-box Chebyshev FMM, uniform quadtree):
//    charges  : gather x (caller order) into sorted per-element DD vectors
//    self     : each element on its own midpoint, FP64 closed form
//    P2M      : W_m = sum_j int_elem b_j S_n(ybar_m, y(s)) ds    (leaves)
//    M2M      : W^parent += S_n(ybar^I, ybar^J) W^J            (upward)
//    M2L      : g^I = sum_{J in IntList(I)} K(xbar^I, ybar^J) W^J   (levels >= 2)
//    L2L      : f^child = g^child + S_n(xbar^child, xbar^parent) f^parent
//    leaf     : L2P + P2P over the neighbour leaves (closed-form element
//               integrals near, Gauss points of the point kernel far)
//  Dense path: every (target, source) pair on the fly (conventional PDDM).
//
// Charges are 4 components per element: potency density sym(D (x) n) (3)
// and fluid source q; potentials are global (sxx, syy, sxy, p), rotated to
// the target element frame at the end.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "kernel_math.cuh"

namespace {

constexpr int MAXGL = 16;
// Quadrature and Chebyshev tables for every supported order, uploaded once
// per device: contexts with different orders can run side by side.
struct GLTab {
    float xn[MAXGL + 1][MAXGL], wn[MAXGL + 1][MAXGL];   // near rule (fluid source), [points][i]
    float xc[DDM_MAX_CHEB / 2][DDM_MAX_CHEB], wc[DDM_MAX_CHEB / 2][DDM_MAX_CHEB];   // P2M rule, n points, [n/2-1]
    float cheb[DDM_MAX_CHEB / 2][DDM_MAX_CHEB], bw[DDM_MAX_CHEB / 2][DDM_MAX_CHEB]; // roots of T_n, barycentric weights
    double x8[8], w8[8];                                 // 8-point Gauss-Legendre rule in FP64 (exact products)
};
__constant__ GLTab c_gl;

// dispatch on the (even) number of Chebyshev nodes per dimension
#define DDM_CHEB_SWITCH(n, M)              \
    switch (n) {                           \
        case 2: M(2); break;               \
        case 4: M(4); break;               \
        case 6: M(6); break;               \
        case 8: M(8); break;               \
        case 10: M(10); break;             \
        case 12: M(12); break;             \
        case 14: M(14); break;             \
        default: M(16); break;             \
    }

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on P_n), FP64 on the host.
void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = n * (z * p1 - p0) / (z * z - 1);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-15) break;
        }
        x[i] = z;
        w[i] = 2 / ((1 - z * z) * dp * dp);
    }
}

// ------------------------------------------------ charges + own element
// Element i (sorted order): its DD vector in the global frame for the
// expansions and the near field, and its own-element term through the
// cached FP64 3x3 block of the time window (caller order).
__device__ __forceinline__ void prep_elem(int64_t i, const double *x, const int64_t *perm, const float4 *frame,
                                          const double *blk, int64_t n, double scale, int overwrite, float4 *chg,
                                          double *y) {
    int64_t e = perm[i];
    float4 f = frame[i];
    double a = x[e], b = x[n + e], c = x[2 * n + e];
    float Ds = (float)a, Dn = (float)b;
    // D = Ds t + Dn n, n = (-ty, tx)
    chg[i] = make_float4(Ds * f.x - Dn * f.y, Ds * f.y + Dn * f.x, (float)c, 0.f);
    const double *B = blk + 9 * e;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        double v = scale * (B[3 * r] * a + B[3 * r + 1] * b + B[3 * r + 2] * c);
        if (overwrite) y[r * n + e] = v; else y[r * n + e] += v;
    }
}

__global__ void k_prep(const double *x, const int64_t *perm, const float4 *frame, const double *blk, int64_t n,
                       double scale, int overwrite, float4 *chg, double *y, float *Wz, float *Fz, int64_t nz) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) prep_elem(i, x, perm, frame, blk, n, scale, overwrite, chg, y);
    // zero the weights and local expansions of the cells above the leaves
    // (the upward pass adds into them)
    for (int64_t z = i; z < nz; z += (int64_t)gridDim.x * blockDim.x) {
        Wz[z] = 0.f;
        Fz[z] = 0.f;
    }
}

// --------------------------------------------------------- own element (FP64)
// own 3x3 blocks (rows sigma_s, sigma_n, p; columns Ds, Dn, Dq), caller order
__global__ void k_self_blocks(KConst<double> k, Win<double> w, const double *xy, int64_t n, double *blk) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double dx = xy[2 * n + e] - xy[e], dy = xy[3 * n + e] - xy[n + e];
    double L = hypot(dx, dy);
    for (int c = 0; c < 3; ++c) {
        double o[3];
        self_field(k, w, 0.5 * L, dx / L, dy / L, c == 0, c == 1, c == 2, o);
        for (int r = 0; r < 3; ++r) blk[9 * e + 3 * r + c] = o[r];
    }
}

// ------------------------------------------------------- upward pass (fused)
// Chebyshev cardinal functions of one point into a strided shared-memory
// column (the approximate divide is well inside the expansion error).
template <int N>
__device__ __forceinline__ void cardinal_col(float x, float *col, int stride) {
    float v[N], s = 0.f;
    int hit = -1;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float d = x - c_gl.cheb[N / 2 - 1][j];
        if (fabsf(d) < 1e-7f) hit = j;
        v[j] = __fdividef(c_gl.bw[N / 2 - 1][j], d);
        s += v[j];
    }
    float is = __fdividef(1.f, s);
#pragma unroll
    for (int j = 0; j < N; ++j) col[j * stride] = hit >= 0 ? (j == hit ? 1.f : 0.f) : v[j] * is;
}

constexpr int UP_T = 256, UP_W = UP_T / 32;
// shared-memory floats of the upward pass: the P2M staging (cardinals of
// UP_T points in x and y, UP_T point weights), the warps' partial weights
// and the M2M staging (leaf weights and their half-transferred copy) share
// one buffer
template <int N>
struct UpSmem {
    static constexpr int N2 = N * N, NOUT = 4 * N2, SXS = UP_T + 1;
    static constexpr int P2M = 2 * N * SXS + 4 * UP_T;
    static constexpr int M2M = 2 * NOUT;
    static constexpr int RED = UP_W * NOUT;
    static constexpr int SIZE = (P2M > M2M ? P2M : M2M) > RED ? (P2M > M2M ? P2M : M2M) : RED;
};

// One block per work item, a chunk of at most ~1024 Gauss points of one leaf
// (large leaves take several blocks, so no block is much longer than the
// rest): P2M of the chunk (paper Sec. 3.3: W_m = sum_j int S_n(ybar_m, y)
// b_j ds, Gauss rule with n points per element, exact for the polynomial
// cardinals) added into the leaf's weights, then the chunk's share of every
// ancestor's weights down to level 2 (M2M), all atomically: the charge
// kernel zeroed the weights and local expansions of every cell of levels
// >= 2.  A leaf above level 2 has no far field and is skipped.
//
// P2M: lane owns node entries (a, b) = lane + 32 j and all 4 components;
// the UP_W warps take every UP_W-th point and are summed at the end.
template <int N>
__device__ __forceinline__ void up_body(const int4 *items, const int2 *leaf_at, float h0, const int32_t *cix,
                                        const int32_t *ciy, const int32_t *parent, const float4 *grel,
                                        const float4 *frame, const float4 *chg, float *W, const float *T,
                                        int64_t bid) {
    using S = UpSmem<N>;
    constexpr int N2 = S::N2, NOUT = S::NOUT, SXS = S::SXS, NE = (N2 + 31) / 32, KO = (NOUT + UP_T - 1) / UP_T;
    __shared__ __align__(16) float sm[S::SIZE];
    __shared__ float sT0[N * N], sT1[N * N];   // child -> parent transfer of the lower and upper half
    float *sx = sm, *sy = sm + N * SXS;
    float4 *wd = reinterpret_cast<float4 *>(sm + 2 * N * SXS);   // 16-byte aligned: 2 N SXS is a multiple of 4
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int4 it = items[bid];               // (leaf, first element, end)
    const int2 la = leaf_at[it.x];            // the leaf's cell and level
    const int64_t leaf = la.x;
    const int L = la.y;
    if (L < 2) return;                        // (the whole block)
    const float hL = ldexpf(h0, -L);          // the leaf's half-width
    const int s0 = it.y, s1 = it.z;
    constexpr int nq = N;                     // Gauss points per element
    float acc[NE][4];
#pragma unroll
    for (int j = 0; j < NE; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const float ih = 1.f / hL;
    const int npts = (s1 - s0) * nq;
    for (int base = 0; base < npts; base += UP_T) {
        int p = base + tid;
        if (p < npts) {
            int e = s0 + p / nq, g = p % nq;
            float4 r = grel[e], f = frame[e], c = chg[e];
            float xi = c_gl.xc[N / 2 - 1][g];
            float px = 0.5f * (r.x + r.z) + xi * f.z * f.x, py = 0.5f * (r.y + r.w) + xi * f.z * f.y;
            cardinal_col<N>(px * ih, sx + tid, SXS);
            cardinal_col<N>(py * ih, sy + tid, SXS);
            float wt = c_gl.wc[N / 2 - 1][g] * f.z;   // ds = a dxi
            float nx = -f.y, ny = f.x;
            wd[tid] = make_float4(wt * c.x * nx, wt * c.y * ny, wt * 0.5f * (c.x * ny + c.y * nx), wt * c.z);
        }
        __syncthreads();
        int np = min(UP_T, npts - base);
        for (int q = warp; q < np; q += UP_W) {
            float4 w4 = wd[q];
#pragma unroll
            for (int j = 0; j < NE; ++j) {
                int ent = lane + 32 * j;
                if (ent < N2) {
                    float v = sx[(ent / N) * SXS + q] * sy[(ent % N) * SXS + q];
                    acc[j][0] = fmaf(v, w4.x, acc[j][0]);
                    acc[j][1] = fmaf(v, w4.y, acc[j][1]);
                    acc[j][2] = fmaf(v, w4.z, acc[j][2]);
                    acc[j][3] = fmaf(v, w4.w, acc[j][3]);
                }
            }
        }
        __syncthreads();
    }
    // sum the warps' partial weights (staging reused)
    float *red = sm;
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        int ent = lane + 32 * j;
        if (ent < N2)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[warp * NOUT + c * N2 + ent] = acc[j][c];
    }
    __syncthreads();
    float *Wc = W + leaf * NOUT;
    float wv[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        int o = tid + k * UP_T;
        wv[k] = 0.f;
        if (o < NOUT) {
#pragma unroll
            for (int w = 0; w < UP_W; ++w) wv[k] += red[w * NOUT + o];
            atomicAdd(Wc + o, wv[k]);
        }
    }
    // M2M up the chain of ancestors down to level 2: the chunk's
    // contribution takes one child -> parent transfer per level (T[q][a][a'],
    // q = the child's half in x and in y, the same tables as L2L) and is
    // added atomically into each ancestor, so no block waits for another.
    // Composed, the transfers are the direct leaf -> ancestor interpolation,
    // exactly.
    float *lw = sm + NOUT, *tmp = sm;          // running contribution, scratch
    __syncthreads();                           // the warp partials are read
#pragma unroll
    for (int k = 0; k < KO; ++k)
        if (tid + k * UP_T < NOUT) lw[tid + k * UP_T] = wv[k];
    for (int e = tid; e < N * N; e += UP_T) {
        sT0[e] = T[e];
        sT1[e] = T[N * N + e];
    }
    int64_t child = leaf;
    for (int l = L - 1; l >= 2; --l) {
        const int64_t anc = parent[child];
        const float *Tx = (cix[child] & 1) ? sT1 : sT0, *Ty = (ciy[child] & 1) ? sT1 : sT0;
        __syncthreads();                           // lw (and the tables) written
        // tmp[c][a][b'] = sum_a' Tx[a][a'] lw[c][a'][b'];  out = sum_b' Ty[b][b'] tmp[c][a][b']
        for (int i = tid; i < NOUT; i += UP_T) {
            const int c = i / N2, aa = (i / N) % N, bb = i % N;
            const float *src = lw + c * N2 + bb;
            float sacc = 0.f;
#pragma unroll
            for (int kk = 0; kk < N; ++kk) sacc = fmaf(Tx[aa * N + kk], src[kk * N], sacc);
            tmp[i] = sacc;
        }
        __syncthreads();
        float o[KO];
#pragma unroll
        for (int kk = 0; kk < KO; ++kk) {
            const int oi = tid + kk * UP_T;
            float sacc = 0.f;
            if (oi < NOUT) {
                const int c = oi / N2, aa = (oi / N) % N, bb = oi % N;
                const float *tc = tmp + c * N2 + aa * N;
#pragma unroll
                for (int j = 0; j < N; ++j) sacc = fmaf(Ty[bb * N + j], tc[j], sacc);
            }
            o[kk] = sacc;
        }
        float *Wa = W + anc * NOUT;
#pragma unroll
        for (int kk = 0; kk < KO; ++kk) {
            const int oi = tid + kk * UP_T;
            if (oi < NOUT) {
                lw[oi] = o[kk];
                atomicAdd(Wa + oi, o[kk]);
            }
        }
        child = anc;
    }
}
template <int N>
__global__ void __launch_bounds__(UP_T) k_up(const int4 *items, const int2 *leaf_at, float h0, const int32_t *cix,
                                             const int32_t *ciy, const int32_t *parent, const float4 *grel,
                                             const float4 *frame, const float4 *chg, float *W, const float *T) {
    up_body<N>(items, leaf_at, h0, cix, ciy, parent, grel, frame, chg, W, T, blockIdx.x);
}

// ----------------------------------------------------- downward pass (fused)
// One block per leaf: f = g at the level-2 ancestor, then down the chain
// f <- S_n(xbar^child, xbar^parent) f + g^child (paper Sec. 3.3 L2L), and
// the leaf's complete local expansion replaces its own M2L sum.  The
// ancestors' values are only read, so leaves sharing them need no order.
// Then L2P at the leaf's targets, four lanes per target (one per component
// of the global sxx, syy, sxy, p).  With y null the four components go to
// far4 (rotated and added after the join); otherwise they are rotated to
// the target frame here and added into y with atomics (the near field, on
// the other stream, adds into y atomically too).
constexpr int L2L_T = 128;
template <int N>
__device__ __forceinline__ void down_body(const int2 *leaf_at, float h0, const int32_t *cix, const int32_t *ciy,
                                          const int32_t *parent, const float *T, const float *F,
                                          const int32_t *cstart, const int32_t *cend, const float4 *grel,
                                          float4 *far4, const float4 *frame, const int64_t *perm, int64_t Ntot,
                                          double scale, double *y, int64_t bid) {
    constexpr int N2 = N * N, NOUT = 4 * N2, KO = (NOUT + L2L_T - 1) / L2L_T;
    constexpr int SP = N2 + 1;                // component stride of sf (padded: the L2P lanes of one target
                                              // read the four components in different banks)
    __shared__ float sT[2 * N2], sf[4 * SP], tmp[NOUT];
    __shared__ int64_t anc[DDM_MAX_LEVELS + 1];
    __shared__ int squad[DDM_MAX_LEVELS + 1];
    const int tid = threadIdx.x;
    const int2 la = leaf_at[bid];             // the leaf's cell and level
    const int64_t leaf = la.x;
    const int L = la.y;
    if (tid == 0) {
        int64_t c = leaf;
        for (int l = L; l >= 2; --l) {
            anc[l] = c;
            squad[l] = ((cix[c] & 1) ? 1 : 0) | ((ciy[c] & 1) ? 2 : 0);
            c = parent[c];
        }
    }
    for (int i = tid; i < 2 * N2; i += L2L_T) sT[i] = T[i];
    __syncthreads();
    // (a leaf above level 2 has no far field: no cell there has an M2L list)
    const float *F2 = L >= 2 ? F + anc[2] * NOUT : nullptr;
    for (int i = tid; i < NOUT; i += L2L_T) sf[(i / N2) * SP + i % N2] = F2 ? F2[i] : 0.f;
    __syncthreads();
    for (int l = 3; l <= L; ++l) {
        const float *Fc = F + anc[l] * NOUT;
        float g[KO];                          // this level's M2L sums, fetched early
#pragma unroll
        for (int k = 0; k < KO; ++k) g[k] = (tid + k * L2L_T < NOUT) ? Fc[tid + k * L2L_T] : 0.f;
        const float *Tx = sT + ((squad[l] & 1) ? N2 : 0), *Ty = sT + ((squad[l] & 2) ? N2 : 0);
        // tmp[c][a'][b] = sum_a Tx[a][a'] f[c][a][b]
        for (int i = tid; i < NOUT; i += L2L_T) {
            int c = i / N2, a = (i / N) % N, b = i % N;
            const float *src = sf + c * SP + b;
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < N; ++k) s = fmaf(Tx[k * N + a], src[k * N], s);
            tmp[i] = s;
        }
        __syncthreads();
        // f[c][a'][b'] = sum_b Ty[b][b'] tmp[c][a'][b] + g
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            int o = tid + k * L2L_T;
            if (o < NOUT) {
                int c = o / N2, a = (o / N) % N, b = o % N;
                const float *tc = tmp + c * N2 + a * N;
                float s = g[k];
#pragma unroll
                for (int j = 0; j < N; ++j) s = fmaf(Ty[j * N + b], tc[j], s);
                sf[c * SP + a * N + b] = s;
            }
        }
        __syncthreads();
    }
    // L2P at the leaf's targets: lane group 4k .. 4k+3 of a warp takes one
    // target, lane c of the group contracts component c
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const float *cheb = c_gl.cheb[N / 2 - 1], *bw = c_gl.bw[N / 2 - 1];
    const float hL = ldexpf(h0, -L);
    const int t0 = cstart[leaf], nt4 = 4 * (cend[leaf] - t0);
    for (int base = 0; base < nt4; base += L2L_T) {   // (the same trip count for the whole block)
        const int w = base + tid, c = w & 3, ti = t0 + (w >> 2);
        const bool on = w < nt4;
        float sum = 0.f;
        if (on) {
            const float4 rt = grel[ti];
            const float xh = __fdividef(0.5f * (rt.x + rt.z), hL), yh = __fdividef(0.5f * (rt.y + rt.w), hL);
            float cx[N], cy[N], sx = 0.f, sy = 0.f;
            int hx = -1, hy = -1;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                float dx = xh - cheb[j], dy = yh - cheb[j];
                if (fabsf(dx) < 1e-7f) hx = j;
                if (fabsf(dy) < 1e-7f) hy = j;
                cx[j] = __fdividef(bw[j], dx);
                cy[j] = __fdividef(bw[j], dy);
                sx += cx[j];
                sy += cy[j];
            }
            const float isx = __fdividef(1.f, sx), isy = __fdividef(1.f, sy);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                cx[j] = hx >= 0 ? (j == hx ? 1.f : 0.f) : cx[j] * isx;
                cy[j] = hy >= 0 ? (j == hy ? 1.f : 0.f) : cy[j] * isy;
            }
            const float *fc = sf + c * SP;
#pragma unroll
            for (int a = 0; a < N; ++a) {
                float row = 0.f;
#pragma unroll
                for (int b = 0; b < N; ++b) row = fmaf(cy[b], fc[a * N + b], row);
                sum = fmaf(cx[a], row, sum);
            }
        }
        const int lb = (tid & 31) & ~3;       // the group's first lane
        const float g0 = __shfl_sync(FULL, sum, lb), g1 = __shfl_sync(FULL, sum, lb + 1);
        const float g2 = __shfl_sync(FULL, sum, lb + 2), g3 = __shfl_sync(FULL, sum, lb + 3);
        if (!on) continue;
        if (!y) {
            if (c == 0) far4[ti] = make_float4(g0, g1, g2, g3);
        } else if (c < 3) {                   // rows sigma_s, sigma_n, p of the target
            float v = g3;
            if (c < 2) {
                const float4 f = frame[ti];
                const float g[4] = {g0, g1, g2, g3};
                float ss, sn;
                to_local<float>(f.x, f.y, g, ss, sn);
                v = c ? sn : ss;
            }
            atomicAdd(y + c * Ntot + perm[ti], scale * (double)v);
        }
    }
}
template <int N>
__global__ void __launch_bounds__(L2L_T) k_down(const int2 *leaf_at, float h0, const int32_t *cix,
                                                const int32_t *ciy, const int32_t *parent, const float *T,
                                                const float *F, const int32_t *cstart, const int32_t *cend,
                                                const float4 *grel, float4 *far4, const float4 *frame,
                                                const int64_t *perm, int64_t Ntot, double scale, double *y) {
    down_body<N>(leaf_at, h0, cix, ciy, parent, T, F, cstart, cend, grel, far4, frame, perm, Ntot, scale, y,
                 blockIdx.x);
}

// ---------------------------------------------------------------------- M2L
// Batched M2L (paper Sec. 3.3 M2L over interaction lists).  The kernel
// between the Chebyshev nodes of two cells depends only on the level, the
// cell offset and the time window, so one (4n^2 x 4n^2) operator per
// (level, offset) is built once per window; the interaction pairs of one
// (level, offset) group then form a GEMM  G = K_{l,o} [W_J1 ... W_JP],
// whose columns are added to the targets' local expansions.
// Operator layout: row (c_out * n^2 + m), column (c_in * n^2 + m').
__global__ void k_m2l_ops(KConst<float> k, Win<float> w, int L, double h0, int n, const int32_t *koff, float *ops) {
    int key = blockIdx.y;
    int lvl = key / 49, o = key % 49, dx = o / 7 - 3, dy = o % 7 - 3;
    if (lvl < 2 || (abs(dx) <= 1 && abs(dy) <= 1) || koff[key + 1] == koff[key]) return;
    int n2 = n * n;
    int np = blockIdx.x * blockDim.x + threadIdx.x;      // node pair (m, m')
    if (np >= n2 * n2) return;
    int m = np / n2, mp = np % n2;
    float h = (float)(h0 / (double)(1 << lvl));
    const float *cheb = c_gl.cheb[(n >> 1) - 1];
    float zx = 2.f * h * dx + h * (cheb[m / n] - cheb[mp / n]);
    float zy = 2.f * h * dy + h * (cheb[m % n] - cheb[mp % n]);
    float *K = ops + (int64_t)key * 16 * n2 * n2;
    int ld = 4 * n2;
    for (int ci = 0; ci < 4; ++ci) {
        float a[4] = {0, 0, 0, 0};
        pot_kernel<float>(k, zx, zy, ci == 0, ci == 1, ci == 2, ci == 3, w, a);
        for (int co = 0; co < 4; ++co) K[(int64_t)(co * n2 + m) * ld + ci * n2 + mp] = a[co];
    }
}

// ------------------------------------------------------ M2L on tcgen05 (TF32)
// The same grouped product G = K_{l,o} [W_J1 ... W_JP] on the fifth-
// generation tensor cores.  One CTA = one work item (column tile of up to
// 64 interaction pairs of one (level, offset) group) x one 128-row slice of
// the 4n^2 operator rows; the 128 x 64 FP32 accumulator lives in tensor
// memory (64 columns).  Operands are split on the way into shared memory,
// x = hi + lo with hi = x with the low 13 mantissa bits cleared (exact in
// TF32) and lo = x - hi (exact in FP32), and each K step issues
// hi*hi + hi*lo + lo*hi (the "3xTF32" product; the dropped lo*lo term is
// ~2^-22 relative), so the result keeps FP32 accuracy.  The four 128-thread
// warps stage K chunks of 32 (one 128-byte row of FP32 per matrix row) into
// a 128-byte-swizzled K-major layout, two stages deep: while the tensor
// core works on one stage, the threads fill the other.  One thread issues
// the MMAs and commits them to the stage's mbarrier.  Every wait is bounded;
// on expiry the CTA raises the context's error word, skips its output and
// still releases its tensor memory.
namespace tc {
constexpr int BM = 128, BN = 64, BK = 32, THREADS = 128, NSTAGE = 2;
constexpr int KSPLIT = 1;                                  // CTAs sharing one tile's K range (sums meet in the atomics)
constexpr int ROWB = BK * 4, CPR = ROWB / 16;             // bytes and 16-byte chunks per tile row
constexpr int A_BYTES = BM * BK * 4, B_BYTES = BN * BK * 4;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // hi and lo of both operands
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;    // + room to align to 1024 B
constexpr uint32_t TMEM_COLS = 64;
constexpr int WAIT_POLLS = 1 << 20;
// instruction descriptor (kind::tf32): D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Tiles are K-major with one ROWB-byte row per matrix row, swizzled in the
// hardware's pattern for that row width: 128-byte rows (BK = 32) XOR the
// 16-byte chunk index with (row mod 8), 1024 B between 8-row groups, swizzle
// mode 2; 64-byte rows (BK = 16) XOR it with (row / 2 mod 4), 512 B between
// 8-row groups, swizzle mode 4.
// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset (unused for swizzled K-major, 16 B), stride byte offset
// (bits 32-45), descriptor version 1 (bit 46), swizzle mode (bits 61-63)
__device__ __forceinline__ uint64_t sw_desc(uint32_t addr) {
    constexpr uint64_t sbo = ROWB == 128 ? 1024 : 512, mode = ROWB == 128 ? 2 : 4;
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46) |
           (mode << 61);
}
// byte offset of 16-byte chunk c of row r in a swizzled tile
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
    return ROWB == 128 ? (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)) : (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

__device__ __forceinline__ void split4(float4 v, float4 &h, float4 &l) {
    h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
    h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
    h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
    h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
    l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with this parity; on expiry set *err (every
// thread keeps the same control flow, so barriers still match)
__device__ __forceinline__ void mbar_wait(uint64_t *bar, uint32_t parity, volatile int *err) {
    if (*err) return;
    for (int i = 0; i < WAIT_POLLS; ++i)
        if (mbar_try(bar, parity)) return;
    *err = 1;
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 TMEM lanes (one per thread of the warp) x 16 consecutive columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
}  // namespace tc

// The grouped gathered product G[:, I] += K_key W[:, J] over the pairs (I, J)
// of one work item, for an operator of M rows and Kd columns per key (at
// ops + key * M * Kd, row-major), sources of stride Kd and targets of stride
// M.  The M2L of a product is M = Kd = 4 n^2; the compressed M2L uses the
// same body for its three stages (bases and cores of other shapes).
__device__ __forceinline__ void tc_group_body(const int2 *work, const int32_t *koff, const int2 *pairs, int M, int Kd,
                                              const float *ops, const float *W, float *F, int *err, int64_t wi) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar[NSTAGE];
    __shared__ uint32_t s_tmem;
    __shared__ int sI[BN], sJ[BN];
    __shared__ int s_err;
    volatile int *verr = &s_err;
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 wk = work[wi];
    const int key = wk.x, p0 = wk.y, p1 = min(koff[key + 1], p0 + BN);
    const int r0 = blockIdx.y * BM;
    const float *K = ops + (int64_t)key * M * Kd;
    if (tid < BN) {
        int p = p0 + tid;
        sI[tid] = p < p1 ? pairs[p].x : -1;
        sJ[tid] = p < p1 ? pairs[p].y : -1;
    }
    if (tid == 0) {
        s_err = 0;
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;
    // this CTA's share of the K chunks
    const int nkt = (Kd + BK - 1) / BK, per = (nkt + (int)gridDim.z - 1) / (int)gridDim.z;
    const int kbeg = blockIdx.z * per, nkb = max(0, min(nkt, kbeg + per) - kbeg);
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % NSTAGE;
        uint8_t *a_hi = base + st * STAGE_BYTES, *a_lo = a_hi + A_BYTES, *b_hi = a_lo + A_BYTES,
                *b_lo = b_hi + B_BYTES;
        const int k0 = (kbeg + kb) * BK;
        constexpr int NA = BM * CPR / THREADS, NB = BN * CPR / THREADS;   // float4 per thread
        float4 va[NA], vb[NB];
#pragma unroll
        for (int i = 0; i < NA; ++i) {       // operator rows r0.., CPR float4 per K chunk
            int idx = tid + i * THREADS, row = idx / CPR, c = idx % CPR, gr = r0 + row, gk = k0 + 4 * c;
            va[i] = (gr < M && gk < Kd) ? __ldg(reinterpret_cast<const float4 *>(K + (int64_t)gr * Kd + gk))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {       // source weights, one column per pair
            int idx = tid + i * THREADS, col = idx / CPR, c = idx % CPR, J = sJ[col], gk = k0 + 4 * c;
            vb[i] = (J >= 0 && gk < Kd) ? __ldg(reinterpret_cast<const float4 *>(W + (int64_t)J * Kd + gk))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // the MMAs that last read this stage (issued NSTAGE chunks ago) must be done
        if (kb >= NSTAGE) mbar_wait(&bar[st], (uint32_t)((kb / NSTAGE - 1) & 1), verr);
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            int idx = tid + i * THREADS, row = idx / CPR, c = idx % CPR;
            float4 h, l;
            split4(va[i], h, l);
            uint32_t off = sw_off(row, c);
            *reinterpret_cast<float4 *>(a_hi + off) = h;
            *reinterpret_cast<float4 *>(a_lo + off) = l;
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            int idx = tid + i * THREADS, col = idx / CPR, c = idx % CPR;
            float4 h, l;
            split4(vb[i], h, l);
            uint32_t off = sw_off(col, c);
            *reinterpret_cast<float4 *>(b_hi + off) = h;
            *reinterpret_cast<float4 *>(b_lo + off) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // stores visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {   // K = 8 per MMA: 32 bytes along the swizzled row
                const uint32_t o = 32u * kk;
                mma_tf32(tmem, sw_desc(al + o), sw_desc(bh + o), (kb | kk) != 0);
                mma_tf32(tmem, sw_desc(ah + o), sw_desc(bl + o), 1u);
                mma_tf32(tmem, sw_desc(ah + o), sw_desc(bh + o), 1u);
            }
            mma_commit(&bar[st]);
        }
    }
    // all MMAs done (the last commit covers every earlier one of the thread)
    if (nkb > 0) mbar_wait(&bar[(nkb - 1) % NSTAGE], (uint32_t)(((nkb - 1) / NSTAGE) & 1), verr);
    fence_after_sync();
    const int row = r0 + warp * 32 + lane;
    const bool ok = *verr == 0 && nkb > 0;
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (ok && row < M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                int I = sI[c0 + j];
                if (I >= 0) atomicAdd(&F[(int64_t)I * M + row], v[j]);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    if (tid == 0 && *verr) atomicExch(err, 1);
}
__device__ __forceinline__ void m2l_body(const int2 *work, const int32_t *koff, const int2 *pairs, int n,
                                         const float *ops, const float *W, float *F, int *err, int64_t wi) {
    tc_group_body(work, koff, pairs, 4 * n * n, 4 * n * n, ops, W, F, err, wi);
}
__global__ void __launch_bounds__(tc::THREADS) k_m2l_tc(const int2 *work, const int32_t *koff, const int2 *pairs,
                                                        int n, const float *ops, const float *W, float *F,
                                                        int *err) {
    m2l_body(work, koff, pairs, n, ops, W, F, err, blockIdx.x);
}
// the same for operators of M x Kd (compressed M2L stages)
__global__ void __launch_bounds__(tc::THREADS) k_tc_group(const int2 *work, const int32_t *koff, const int2 *pairs,
                                                          int M, int Kd, const float *ops, const float *W, float *F,
                                                          int *err) {
    tc_group_body(work, koff, pairs, M, Kd, ops, W, F, err, blockIdx.x);
}

// ----------------------------------------------------------- leaf L2P + P2P
struct SrcTile {
    float x0, y0, x1, y1;      // end points in the target leaf frame
    float Dx, Dy, q, a;        // DD vector, source strength, half-length
    float tx, ty;              // tangent
    int idx;                   // sorted index
};

__device__ __forceinline__ void q_point(const KConst<float> &k, float zx, float zy, float q, const Win<float> &w,
                                        float acc[4]) {
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        float ct = side == 0 ? w.ct_hi : w.ct_lo;
        if (ct <= 0.f) continue;
        float s = side == 0 ? 1.f : -1.f;
        float x2 = zx * zx, y2 = zy * zy, r2 = x2 + y2;
        float ir2 = __fdividef(1.f, r2);
        float g0c = side == 0 ? w.g_hi : w.g_lo;
        float u = r2 * g0c, iu = 4.f * ct * ir2;
        float e, F0, F1, F2;
        f_funcs<float>(u, iu, e, F0, F1, F2);
        float E1 = e1f(u, iu);
        float pre = s * q * k.i4pk, nn = 2.f * F0 * ir2;
        acc[0] -= pre * k.eta * (nn * x2 + E1 - F0);
        acc[1] -= pre * k.eta * (nn * y2 + E1 - F0);
        acc[2] -= pre * k.eta * (nn * zx * zy);
        acc[3] += pre * E1;
    }
}

// Far pairs (centre distance r > 8 a): Gauss-Legendre rule of the point
// kernel along the element.  The m-point rule's relative error for a kernel
// decaying like r^-2 is about c_m (a/r)^(2m) (c_2 ~ 0.44, c_3 ~ 0.16): 3
// points (nodes 0, +-sqrt(3/5), weights 8/9, 5/9) up to r = 24 a (<= 6e-7
// at r = 8 a) and 2 points (+-1/sqrt(3), weights 1) beyond (<= 1.3e-6).
// PRECISE: the DD part in FP64 with the 3-point rule at every distance.
__device__ __forceinline__ void far_node(int ng, int g, float &xi, float &wt) {
    if (ng == 3) {
        xi = g == 0 ? -0.77459666924f : (g == 1 ? 0.f : 0.77459666924f);
        wt = g == 1 ? 0.88888888889f : 0.55555555556f;
    } else {
        xi = g == 0 ? -0.57735026919f : 0.57735026919f;
        wt = 1.f;
    }
}
// A source element as the far-pair rule needs it, built once per source
// and shared by every target: potency per unit length as trace, Pxx - Pyy
// and 2 Pxy (DD vector D, normal n: P = sym(D n)), fluid source,
// half-length and tangent, and the squared distances below which 3 Gauss
// points are taken (24 a) and beyond which every Gauss point is at u > Big
// on both sides of the window ((a + rbig)^2).
struct FarSrc {
    float Pd, P2, Tr, q, a, tx, ty, r2_big, a2tr, a2ti;
};
__device__ __forceinline__ FarSrc far_src(float a, float tx, float ty, float Dx, float Dy, float q, float rbig) {
    const float nx = -ty, ny = tx, pxx = Dx * nx, pyy = Dy * ny, rb = a + rbig, a2 = a * a;
    return FarSrc{pxx - pyy, Dx * ny + Dy * nx, pxx + pyy, q, a, tx, ty, rb * rb, a2 * (tx * tx - ty * ty),
                  2.f * a2 * tx * ty};
}
// FP32 pair from a prepared source, the target at (dx, dy) from its
// midpoint: where u > Big along the whole element (r > a + rbig), the exact
// element integral of the rational kernel (at any distance); otherwise
// (only for r > 8 a) the Gauss rule of the full point kernel
__device__ __forceinline__ void far_pair_f(const KConst<float> &k, const Win<float> &w, float dx, float dy, float r2,
                                           const FarSrc &s, float acc[4]) {
    if (r2 > s.r2_big) {
        const float d4ct = 4.f * (w.ct_hi - w.ct_lo);
        const float ce = w.elastic ? k.Cu : 0.f, pc = w.elastic ? k.pS : 0.f;
        elem_bigu<float>(dx, dy, s.a2tr, s.a2ti, s.a * s.a, 2.f * s.a, s.Pd, s.P2, s.Tr, s.q, ce, pc, k.a6 * d4ct,
                         -k.qe * d4ct, acc);
        return;
    }
    const int ng = r2 <= 576.f * s.a * s.a ? 3 : 2;
    const float Pxx = 0.5f * (s.Tr + s.Pd), Pyy = 0.5f * (s.Tr - s.Pd), Pxy = 0.5f * s.P2;
#pragma unroll 1
    for (int g = 0; g < ng; ++g) {
        float xi, wt;
        far_node(ng, g, xi, wt);
        const float sg = xi * s.a, wg = wt * s.a;
        pot_kernel<float>(k, dx - sg * s.tx, dy - sg * s.ty, wg * Pxx, wg * Pyy, wg * Pxy, wg * s.q, w, acc);
    }
}
template <bool PRECISE>
__device__ __forceinline__ void far_pair(const KConst<float> &k, const KConst<double> &kd, const Win<float> &w,
                                         const Win<double> &wd, float dx, float dy, float r2, float a, float tx,
                                         float ty, float Dx, float Dy, float q, float acc[4], double accd[4]) {
    if (PRECISE) {
        double nx = -(double)ty, ny = (double)tx;
        const double ad = a, rb = ad + wd.rbig;
        if ((double)r2 > rb * rb) {
            // u > Big along the element: the exact rational integral, all in FP64
            const double d4ct = 4.0 * (wd.ct_hi - wd.ct_lo);
            const double pxx = Dx * nx, pyy = Dy * ny;
            const double tdx = tx, tdy = ty;
            elem_bigu<double>(dx, dy, ad * ad * (tdx * tdx - tdy * tdy), 2.0 * ad * ad * tdx * tdy, ad * ad, 2.0 * ad,
                              pxx - pyy, Dx * ny + Dy * nx, pxx + pyy, (double)q, wd.elastic ? kd.Cu : 0.0,
                              wd.elastic ? kd.pS : 0.0, kd.a6 * d4ct, -kd.qe * d4ct, accd);
            return;
        }
        double Pxx = Dx * nx, Pyy = Dy * ny, Pxy = 0.5 * (Dx * ny + Dy * nx);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            float xi, wt;
            far_node(3, g, xi, wt);
            double sg = (double)xi * a, wg = (double)wt * a;
            pot_kernel<double>(kd, dx - sg * tx, dy - sg * ty, wg * Pxx, wg * Pyy, wg * Pxy, 0.0, wd, accd);
            if (q != 0.f) q_point(k, dx - (float)sg * tx, dy - (float)sg * ty, (float)wg * q, w, acc);
        }
        return;
    }
    far_pair_f(k, w, dx, dy, r2, far_src(a, tx, ty, Dx, Dy, q, w.rbig), acc);
}

// Close pairs (r <= 8 a), split into units: unit 0 / 1 = the dislocation
// at end point 0 (+) / 1 (-) (exact element integral of the DD part),
// unit 2 + g = Gauss point g of the nq-point rule for the fluid source.
// (x0, y0, x1, y1) are the source end points and (mx, my) the target in
// the same frame.  PRECISE: the DD units in FP64.
template <bool PRECISE>
__device__ __forceinline__ void near_unit(int unit, int nq, const KConst<float> &k, const KConst<double> &kd,
                                          const Win<float> &w, const Win<double> &wd, float mx, float my, float x0,
                                          float y0, float x1, float y1, float a, float tx, float ty, float Dx,
                                          float Dy, float q, float acc[4], double accd[4]) {
    if (unit < 2) {
        float ex = unit ? x1 : x0, ey = unit ? y1 : y0;
        if (PRECISE)
            disl_field<double>(kd, (double)(mx - ex), (double)(my - ey), (double)Dx, (double)Dy, wd,
                               unit ? -1.0 : 1.0, accd);
        else
            disl_field<float>(k, mx - ex, my - ey, Dx, Dy, w, unit ? -1.f : 1.f, acc);
    } else if (q != 0.f) {
        int g = unit - 2;
        float sg = c_gl.xn[nq][g] * a, wt = c_gl.wn[nq][g] * a;
        float cx = 0.5f * (x0 + x1), cy = 0.5f * (y0 + y1);
        q_point(k, mx - cx - sg * tx, my - cy - sg * ty, wt * q, w, acc);
    }
}

// one (target, source) pair, self pairs excluded by the caller
template <bool PRECISE>
__device__ __forceinline__ void pair_field(const KConst<float> &k, const KConst<double> &kd, const Win<float> &w,
                                           const Win<double> &wd, int nq, float mx, float my, const SrcTile &s,
                                           float acc[4], double accd[4]) {
    float dx = mx - 0.5f * (s.x0 + s.x1), dy = my - 0.5f * (s.y0 + s.y1);
    float r2 = dx * dx + dy * dy;
    const float rb = s.a + w.rbig;            // beyond: u > Big along the element (exact integral)
    if (r2 > 64.f * s.a * s.a || (!PRECISE && r2 > rb * rb)) {
        far_pair<PRECISE>(k, kd, w, wd, dx, dy, r2, s.a, s.tx, s.ty, s.Dx, s.Dy, s.q, acc, accd);
    } else {
        int nu = 2 + (s.q != 0.f ? nq : 0);
        for (int u = 0; u < nu; ++u)
            near_unit<PRECISE>(u, nq, k, kd, w, wd, mx, my, s.x0, s.y0, s.x1, s.y1, s.a, s.tx, s.ty, s.Dx, s.Dy,
                               s.q, acc, accd);
    }
}

// Near field + L2P.  One warp per target.  The lanes walk the sources of
// the target leaf's neighbour leaves (self + up to 8; table precomputed per
// leaf: start, count, cell offset) 32 at a time and evaluate the far pairs
// at once; close pairs go to a per-warp queue and are evaluated afterwards
// as independent units (2 dislocations + nq fluid-source points each), so
// the costly close-pair arithmetic runs on full warps instead of on the few
// lanes that meet a close pair in each step.  Each lane sums its pairs in
// FP32, the warp then reduces in FP64; L2P is split over the lanes by
// Chebyshev node and reduced the same way.
constexpr int NEAR_W = 8;
constexpr int NEAR_T = 32 * NEAR_W;
constexpr int NEAR_Q = 64;     // close pairs queued per target; further ones are evaluated in place
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
// FP64 runs at 1/64 of the FP32 rate on this GPU, so the per-target sums
// are carried as unevaluated FP32 pairs (h + l, Knuth's two-sum), which
// keeps ~44 bits through the warp reduction at FP32 cost.
__device__ __forceinline__ void two_sum_add(float &h, float &l, float bh, float bl) {
    float s = h + bh, v = s - h;
    float e = (h - (s - v)) + (bh - v) + (l + bl);
    h = s + e;
    l = e - (h - s);
}
__device__ __forceinline__ void warp_sum_ds(float &h, float &l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float bh = __shfl_xor_sync(0xFFFFFFFFu, h, o), bl = __shfl_xor_sync(0xFFFFFFFFu, l, o);
        two_sum_add(h, l, bh, bl);
    }
}
// One chunk (up to 32) of a leaf's direct-interaction records into the
// warp's table: element starts and the prefix sums of the counts (one lane
// per record).
constexpr int REC_CHUNK = 32;
__device__ __forceinline__ void load_recs(const int4 *nbtab, int q, int nc, int lane, int *sst, int *spre) {
    const int4 tb = lane < nc ? nbtab[q + lane] : make_int4(0, 0, 0, 0);
    int incl = tb.y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane < nc) {
        sst[lane] = tb.x;
        spre[lane + 1] = incl;
    }
    if (lane == 0) spre[0] = 0;
}
template <bool PRECISE>
__global__ void __launch_bounds__(NEAR_T, 4) k_near(KConst<float> k, KConst<double> kd, Win<float> w, Win<double> wd,
                                                 const int32_t *nboff, const int4 *nbtab, const int32_t *elem_leaf,
                                                 const float4 *grel, const float4 *gloc, const float2 *ggrid,
                                                 float g16, const float4 *frame, const float4 *chg,
                                                 const int64_t *perm, const int2 *leaf_at, float h0, int n, int nq,
                                                 const float *F, int use_far, int64_t N, double scale, double *y) {
    constexpr unsigned FULL = 0xFFFFFFFFu;
    __shared__ int sst[NEAR_W][REC_CHUNK], spre[NEAR_W][REC_CHUNK + 1];
    __shared__ int2 sq[NEAR_W][NEAR_Q];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ti = (int64_t)blockIdx.x * NEAR_W + wid;
    if (ti >= N) return;                      // whole warp leaves together
    const int32_t leaf = elem_leaf[ti];
    const int q0 = nboff[leaf], nb = nboff[leaf + 1] - q0;
    // pairs: positions relative to the target's grid point (exact grid
    // differences times g16); L2P: the target relative to its leaf centre
    const float4 lt = gloc[ti];
    const float2 gt = ggrid[ti];
    const float mx = 0.5f * (lt.x + lt.z), my = 0.5f * (lt.y + lt.w);
    // lanes 0, 1, 2 write sigma_s, sigma_n, p at the end: fetch what they need now
    int64_t eout = 0;
    float4 fout = make_float4(0.f, 0.f, 0.f, 0.f);
    double yold = 0.0;
    if (lane < 3) {
        eout = perm[ti];
        fout = frame[ti];
        yold = y[lane * N + eout];
    }
    float acc[4] = {0, 0, 0, 0};
    double accd[4] = {0, 0, 0, 0};
    int qn = 0;
    bool anyq = false;
    for (int cb = 0; cb < nb; cb += REC_CHUNK) {   // records in chunks (a uniform tree has <= 9)
        const int nc = min(REC_CHUNK, nb - cb);
        __syncwarp();                             // the previous chunk's table is read
        load_recs(nbtab, q0 + cb, nc, lane, sst[wid], spre[wid]);
        __syncwarp();
        const int S = spre[wid][nc];
        int slot = 0;
        for (int base = 0; base < S; base += 32) {
            const int c = base + lane;
            bool close = false, hasq = false;
            int sj = -1;
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f), f = r, cg = r;
            float ox = 0.f, oy = 0.f;
            if (c < S) {
                while (c >= spre[wid][slot + 1]) ++slot;
                sj = sst[wid][slot] + (c - spre[wid][slot]);
                if (sj != (int)ti) {
                    r = gloc[sj];
                    f = frame[sj];
                    cg = chg[sj];
                    const float2 gs = ggrid[sj];
                    ox = g16 * (gs.x - gt.x);
                    oy = g16 * (gs.y - gt.y);
                    float dx = mx - 0.5f * (r.x + r.z) - ox, dy = my - 0.5f * (r.y + r.w) - oy;
                    float r2 = dx * dx + dy * dy;
                    if (r2 > 64.f * f.z * f.z)
                        far_pair<PRECISE>(k, kd, w, wd, dx, dy, r2, f.z, f.x, f.y, cg.x, cg.y, cg.z, acc, accd);
                    else {
                        close = true;
                        hasq = cg.z != 0.f;
                    }
                }
            }
            const unsigned m = __ballot_sync(FULL, close);
            if (m) {
                anyq = anyq || __ballot_sync(FULL, hasq) != 0u;
                const int pos = qn + __popc(m & ((1u << lane) - 1u));
                if (close) {
                    if (pos < NEAR_Q) {
                        sq[wid][pos] = make_int2(sj, slot);
                    } else {                      // queue full: this pair in place
                        int nu = 2 + (hasq ? nq : 0);
                        for (int u = 0; u < nu; ++u)
                            near_unit<PRECISE>(u, nq, k, kd, w, wd, mx, my, r.x + ox, r.y + oy, r.z + ox, r.w + oy, f.z,
                                               f.x, f.y, cg.x, cg.y, cg.z, acc, accd);
                    }
                }
                qn += __popc(m);
            }
        }
    }
    __syncwarp();
    const int nqd = qn < NEAR_Q ? qn : NEAR_Q;
    if (nqd > 0) {
        // units: first the 2 dislocations of every queued pair, then the
        // fluid-source points (only if some queued source carries q)
        const int nf = anyq ? nq : 0, nd = 2 * nqd, U = nd + nf * nqd;
        for (int base = 0; base < U; base += 32) {
            const int u = base + lane;
            if (u < U) {
                int pi, unit;
                if (u < nd) {
                    pi = u >> 1;
                    unit = u & 1;
                } else {
                    pi = (u - nd) / nf;
                    unit = 2 + (u - nd) - pi * nf;
                }
                const int2 e = sq[wid][pi];
                const float4 r = gloc[e.x], f = frame[e.x], cg = chg[e.x];
                const float2 gs = ggrid[e.x];
                const float ox = g16 * (gs.x - gt.x), oy = g16 * (gs.y - gt.y);
                near_unit<PRECISE>(unit, nq, k, kd, w, wd, mx, my, r.x + ox, r.y + oy, r.z + ox, r.w + oy, f.z, f.x,
                                   f.y, cg.x, cg.y, cg.z, acc, accd);
            }
        }
    }
    float hl[4][2];                           // per-lane sums as FP32 pairs
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        hl[c][0] = acc[c];
        hl[c][1] = 0.f;
    }
    if (use_far) {
        // L2P.  Barycentric terms: lane j < n takes x node j, lane 16 + j
        // y node j; the sums are reduced within each half-warp, and every
        // lane then fetches the two cardinals of its nodes m = lane,
        // lane + 32, ... by shuffle.
        const float *cheb = c_gl.cheb[(n >> 1) - 1], *bw = c_gl.bw[(n >> 1) - 1];
        const int2 la = leaf_at[leaf];
        const float hL = ldexpf(h0, -la.y);
        const int j = lane & 15;
        const bool isy = lane >= 16;
        float tv = 0.f;
        bool hit = false;
        if (j < n) {
            const float4 rt = grel[ti];
            const float lx = 0.5f * (rt.x + rt.z), ly = 0.5f * (rt.y + rt.w);
            float d = __fdividef(isy ? ly : lx, hL) - cheb[j];
            hit = fabsf(d) < 1e-7f;
            tv = hit ? 0.f : __fdividef(bw[j], d);
        }
        float sum = tv;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
        const unsigned hm = __ballot_sync(FULL, hit);
        const bool half_hit = isy ? (hm >> 16) != 0u : (hm & 0xFFFFu) != 0u;
        const float card = half_hit ? (hit ? 1.f : 0.f) : tv * __fdividef(1.f, sum);
        const int n2 = n * n;
        const float *Fc = F + (int64_t)la.x * 4 * n2;
        float f4[4] = {0, 0, 0, 0};
        for (int base = 0; base < n2; base += 32) {
            const int m = base + lane, mc = m < n2 ? m : n2 - 1;
            const int a = mc / n, bb = mc - a * n;
            const float v = __shfl_sync(FULL, card, a) * __shfl_sync(FULL, card, 16 + bb);
            if (m < n2) {
                f4[0] += v * Fc[m]; f4[1] += v * Fc[n2 + m]; f4[2] += v * Fc[2 * n2 + m]; f4[3] += v * Fc[3 * n2 + m];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) two_sum_add(hl[c][0], hl[c][1], f4[c], 0.f);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) warp_sum_ds(hl[c][0], hl[c][1]);
    if (PRECISE) {                            // the FP64 part of the DD units
#pragma unroll
        for (int c = 0; c < 4; ++c) accd[c] = warp_sum(accd[c]);
    }
    // lanes 0, 1, 2 write sigma_s, sigma_n, p; the rotation to the target
    // frame is applied to both halves of each pair
    if (lane >= 3) return;
    const float4 f = fout;
    const float nx = -f.y, ny = f.x;
    float vh, vl;
    double vd = 0.0;
    if (lane == 2) {
        vh = hl[3][0];
        vl = hl[3][1];
        if (PRECISE) vd = accd[3];
    } else {
        // sigma_n = g . (n n), sigma_s = g . sym(t n)
        const float cxx = lane ? nx * nx : f.x * nx, cyy = lane ? ny * ny : f.y * ny;
        const float cxy = lane ? 2.f * nx * ny : f.x * ny + f.y * nx;
        vh = cxx * hl[0][0] + cyy * hl[1][0] + cxy * hl[2][0];
        vl = cxx * hl[0][1] + cyy * hl[1][1] + cxy * hl[2][1];
        if (PRECISE) vd = (double)cxx * accd[0] + (double)cyy * accd[1] + (double)cxy * accd[2];
    }
    y[lane * N + eout] = yold + scale * (((double)vh + (double)vl) + vd);
}

// Near field for two targets per warp (non-precise products): a work item is
// a pair of consecutive targets of one leaf (or a single), so the two share
// the neighbour table, the walk over the sources and every source load,
// and each warp carries twice the independent work through the same chain
// of dependent loads.  Close pairs are queued per (source, target) and
// evaluated afterwards as units, as in k_near.  L2P runs separately
// (k_l2p).
// TWO: the window may start after 0 (history terms); otherwise t_lo = 0 is
// known at compile time and the two-sided code paths drop out of the kernel
template <bool TWO>
__device__ __forceinline__ void near2_body(const KConst<float> &k, const Win<float> &win, const int32_t *nboff,
                                           const int4 *nbtab, const int32_t *elem_leaf, const float4 *gloc,
                                           const float2 *ggrid, const float4 *frame, const float4 *chg,
                                           const int64_t *perm, float g16, int nq, const int2 *items, int64_t N,
                                           double scale, double *y, int64_t item) {
    const Win<float> w = TWO ? win : Win<float>{win.ct_hi, 0.f, win.g_hi, 0.f, 1, win.rbig};
    constexpr unsigned FULL = 0xFFFFFFFFu;
    __shared__ int sst[NEAR_W][REC_CHUNK], spre[NEAR_W][REC_CHUNK + 1];
    __shared__ int2 sq[NEAR_W][NEAR_Q];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 it = items[item];
    const int t0 = it.x, t1 = it.y >= 0 ? it.y : it.x;
    const bool two = it.y >= 0;
    const int32_t leaf = elem_leaf[t0];
    const int q0 = nboff[leaf], nb = nboff[leaf + 1] - q0;
    // every position below is relative to target 0's grid point: an
    // element's own offset from its grid point plus the exact grid
    // difference times g16 (rounded once, relative to the distance)
    const float4 ra = gloc[t0], rb = gloc[t1];
    const float2 ga = ggrid[t0], gb = ggrid[t1];
    const float mx0 = 0.5f * (ra.x + ra.z), my0 = 0.5f * (ra.y + ra.w);
    const float mx1 = fmaf(gb.x - ga.x, g16, 0.5f * (rb.x + rb.z)), my1 = fmaf(gb.y - ga.y, g16, 0.5f * (rb.y + rb.w));
    // lanes 0-2 write target 0's rows, lanes 3-5 target 1's: fetch what they need now
    const bool writer = lane < 3 || (two && lane < 6);
    const int tw = lane < 3 ? t0 : t1, row = lane < 3 ? lane : lane - 3;
    int64_t eout = 0;
    float4 fout = make_float4(0.f, 0.f, 0.f, 0.f);
    if (writer) {
        eout = perm[tw];
        fout = frame[tw];
    }
    float acc0[4] = {0, 0, 0, 0}, acc1[4] = {0, 0, 0, 0};
    double dummy[4];
    int qn = 0;
    bool anyq = false;
    for (int cb = 0; cb < nb; cb += REC_CHUNK) {   // records in chunks (a uniform tree has <= 9)
        const int nc = min(REC_CHUNK, nb - cb);
        __syncwarp();                             // the previous chunk's table is read
        load_recs(nbtab, q0 + cb, nc, lane, sst[wid], spre[wid]);
        __syncwarp();
        const int S = spre[wid][nc];
        int slot = 0;
        for (int base = 0; base < S; base += 32) {
            const int c = base + lane;
            bool close0 = false, close1 = false, hasq = false;
            int sj = -1;
            if (c < S) {
                while (c >= spre[wid][slot + 1]) ++slot;
                sj = sst[wid][slot] + (c - spre[wid][slot]);
                const float4 r = gloc[sj], f = frame[sj], cg = chg[sj];
                const float2 gs = ggrid[sj];
                const float cxs = fmaf(gs.x - ga.x, g16, 0.5f * (r.x + r.z)), cys = fmaf(gs.y - ga.y, g16, 0.5f * (r.y + r.w));
                const float lim = 64.f * f.z * f.z;
                const FarSrc fs = far_src(f.z, f.x, f.y, cg.x, cg.y, cg.z, w.rbig);
                hasq = cg.z != 0.f;
                // beyond 8 a, or anywhere u > Big along the element: at once
                const float lim2 = fminf(lim, fs.r2_big);
                if (sj != t0) {
                    const float dx = mx0 - cxs, dy = my0 - cys, r2 = dx * dx + dy * dy;
                    if (r2 > lim2) far_pair_f(k, w, dx, dy, r2, fs, acc0);
                    else close0 = true;
                }
                if (two && sj != t1) {
                    const float dx = mx1 - cxs, dy = my1 - cys, r2 = dx * dx + dy * dy;
                    if (r2 > lim2) far_pair_f(k, w, dx, dy, r2, fs, acc1);
                    else close1 = true;
                }
            }
            // queue the close (source, target) pairs: entry (source, slot | target << 8)
#pragma unroll
            for (int tg = 0; tg < 2; ++tg) {
                const bool cl = tg ? close1 : close0;
                const unsigned m = __ballot_sync(FULL, cl);
                if (m) {
                    anyq = anyq || __ballot_sync(FULL, cl && hasq) != 0u;
                    const int pos = qn + __popc(m & ((1u << lane) - 1u));
                    if (cl) {
                        if (pos < NEAR_Q) {
                            sq[wid][pos] = make_int2(sj, slot | (tg << 8));
                        } else {                  // queue full: this pair in place
                            const float4 r = gloc[sj], f = frame[sj], cg = chg[sj];
                            const float2 gs = ggrid[sj];
                            const float ox = g16 * (gs.x - ga.x), oy = g16 * (gs.y - ga.y);
                            const int nu = 2 + (cg.z != 0.f ? nq : 0);
                            float a4[4] = {0, 0, 0, 0};
                            for (int u = 0; u < nu; ++u)
                                near_unit<false>(u, nq, k, KConst<double>{}, w, Win<double>{}, tg ? mx1 : mx0,
                                                 tg ? my1 : my0, r.x + ox, r.y + oy, r.z + ox, r.w + oy, f.z, f.x, f.y,
                                                 cg.x, cg.y, cg.z, a4, dummy);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                acc0[c] += tg ? 0.f : a4[c];
                                acc1[c] += tg ? a4[c] : 0.f;
                            }
                        }
                    }
                    qn += __popc(m);
                }
            }
        }
    }
    __syncwarp();
    const int nqd = qn < NEAR_Q ? qn : NEAR_Q;
    if (nqd > 0) {
        // units: first the 2 dislocations of every queued pair, then the
        // fluid-source points (only if some queued source carries q)
        const int nf = anyq ? nq : 0, nd = 2 * nqd, U = nd + nf * nqd;
        for (int base = 0; base < U; base += 32) {
            const int u = base + lane;
            if (u < U) {
                int pi, unit;
                if (u < nd) {
                    pi = u >> 1;
                    unit = u & 1;
                } else {
                    pi = (u - nd) / nf;
                    unit = 2 + (u - nd) - pi * nf;
                }
                const int2 e = sq[wid][pi];
                const int tg = e.y >> 8;
                const float4 r = gloc[e.x], f = frame[e.x], cg = chg[e.x];
                const float2 gs = ggrid[e.x];
                const float ox = g16 * (gs.x - ga.x), oy = g16 * (gs.y - ga.y);
                float a4[4] = {0, 0, 0, 0};
                near_unit<false>(unit, nq, k, KConst<double>{}, w, Win<double>{}, tg ? mx1 : mx0, tg ? my1 : my0,
                                 r.x + ox, r.y + oy, r.z + ox, r.w + oy, f.z, f.x, f.y, cg.x, cg.y, cg.z, a4, dummy);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc0[c] += tg ? 0.f : a4[c];
                    acc1[c] += tg ? a4[c] : 0.f;
                }
            }
        }
    }
    float hl[8][2];                           // per-lane sums as FP32 pairs
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        hl[c][0] = acc0[c];
        hl[4 + c][0] = acc1[c];
        hl[c][1] = hl[4 + c][1] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) warp_sum_ds(hl[c][0], hl[c][1]);
    if (!writer) return;
    const int b0 = lane < 3 ? 0 : 4;
    const float4 f = fout;
    const float nx = -f.y, ny = f.x;
    float vh, vl;
    if (row == 2) {
        vh = hl[b0 + 3][0];
        vl = hl[b0 + 3][1];
    } else {
        // sigma_n = g . (n n), sigma_s = g . sym(t n)
        const float cxx = row ? nx * nx : f.x * nx, cyy = row ? ny * ny : f.y * ny;
        const float cxy = row ? 2.f * nx * ny : f.x * ny + f.y * nx;
        vh = cxx * hl[b0][0] + cyy * hl[b0 + 1][0] + cxy * hl[b0 + 2][0];
        vl = cxx * hl[b0][1] + cyy * hl[b0 + 1][1] + cxy * hl[b0 + 2][1];
    }
    // atomically: the far field of the same product may be added beside it
    atomicAdd(y + row * N + eout, scale * ((double)vh + (double)vl));
}
template <bool TWO>
__global__ void __launch_bounds__(NEAR_T, 4) k_near2(KConst<float> k, Win<float> w, const int32_t *nboff,
                                                     const int4 *nbtab, const int32_t *elem_leaf, const float4 *gloc,
                                                     const float2 *ggrid, const float4 *frame, const float4 *chg,
                                                     const int64_t *perm, float g16, int nq, const int2 *items,
                                                     int64_t n_items, int64_t N, double scale, double *y) {
    const int64_t item = (int64_t)blockIdx.x * NEAR_W + (threadIdx.x >> 5);
    if (item >= n_items) return;              // whole warp leaves together
    near2_body<TWO>(k, w, nboff, nbtab, elem_leaf, gloc, ggrid, frame, chg, perm, g16, nq, items, N, scale, y, item);
}

// far field at the targets (from k_down) rotated to each target frame and
// added: y += scale * (sigma_s, sigma_n, p)
__global__ void k_far_add(const float4 *far4, const float4 *frame, const int64_t *perm, int64_t Ntot, double scale,
                          double *y) {
    const int64_t ti = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ti >= Ntot) return;
    const float4 g4 = far4[ti], f = frame[ti];
    const float g[4] = {g4.x, g4.y, g4.z, g4.w};
    float ss, sn;
    to_local<float>(f.x, f.y, g, ss, sn);
    const int64_t e = perm[ti];
    y[e] += scale * (double)ss;
    y[Ntot + e] += scale * (double)sn;
    y[2 * Ntot + e] += scale * (double)g4.w;
}

// -------------------------------------------------------------------- dense
constexpr int DN_T = 128;
template <bool PRECISE>
__global__ void __launch_bounds__(DN_T) k_dense(KConst<float> k, KConst<double> kd, Win<float> w, Win<double> wd,
                                                int nq, const float4 *gloc, const float2 *ggrid, float g16,
                                                const float4 *frame, const float4 *chg, const int64_t *perm,
                                                int64_t N, int64_t chunk, double scale, double *y) {
    __shared__ SrcTile tile[DN_T];
    __shared__ float sgx[DN_T], sgy[DN_T];
    int64_t ti = blockIdx.x * (int64_t)DN_T + threadIdx.x;
    bool act = ti < N;
    float mx = 0, my = 0, ttx = 1, tty = 0;
    float gtx = 0.f, gty = 0.f;
    if (act) {                                // positions relative to the target's grid point
        float4 r = gloc[ti], f = frame[ti];
        mx = 0.5f * (r.x + r.z); my = 0.5f * (r.y + r.w);
        ttx = f.x; tty = f.y;
        const float2 g = ggrid[ti];
        gtx = g.x; gty = g.y;
    }
    double accd[4] = {0, 0, 0, 0};
    int64_t s0 = blockIdx.y * chunk;
    int64_t s1 = s0 + chunk < N ? s0 + chunk : N;
    for (int64_t sb = s0; sb < s1; sb += DN_T) {
        __syncthreads();
        int64_t sj = sb + threadIdx.x;
        if (sj < s1) {
            float4 r = gloc[sj], f = frame[sj], c = chg[sj];
            SrcTile s;
            s.x0 = r.x; s.y0 = r.y; s.x1 = r.z; s.y1 = r.w;
            s.Dx = c.x; s.Dy = c.y; s.q = c.z; s.a = f.z; s.tx = f.x; s.ty = f.y; s.idx = (int)sj;
            tile[threadIdx.x] = s;
            const float2 g = ggrid[sj];
            sgx[threadIdx.x] = g.x;
            sgy[threadIdx.x] = g.y;
        }
        __syncthreads();
        int cnt = (int)(s1 - sb < DN_T ? s1 - sb : DN_T);
        if (act) {
            float acc[4] = {0, 0, 0, 0};          // one tile in FP32, tiles summed in FP64
            for (int j = 0; j < cnt; ++j) {
                if (tile[j].idx == (int)ti) continue;
                SrcTile s = tile[j];
                const float ox = g16 * (sgx[j] - gtx), oy = g16 * (sgy[j] - gty);
                s.x0 += ox; s.y0 += oy; s.x1 += ox; s.y1 += oy;
                pair_field<PRECISE>(k, kd, w, wd, nq, mx, my, s, acc, accd);
            }
            for (int c = 0; c < 4; ++c) accd[c] += (double)acc[c];
        }
    }
    if (act) {
        double ss, sn;
        to_local<double>((double)ttx, (double)tty, accd, ss, sn);
        int64_t e = perm[ti];
        atomicAdd(&y[e], scale * ss);
        atomicAdd(&y[N + e], scale * sn);
        atomicAdd(&y[2 * N + e], scale * accd[3]);
    }
}

// Fluid source at a point in FP64 (both sides of the window), the q terms of
// the point kernel: p = Q E1(u) / (4 pi kappa),
// sigma = -(eta Q / (4 pi kappa)) (2 F n n + (E1 - F) I).
__device__ __forceinline__ void q_point_d(const KConst<double> &k, double zx, double zy, double q,
                                          const Win<double> &w, double acc[4]) {
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const double ct = side == 0 ? w.ct_hi : w.ct_lo;
        if (ct <= 0.0) continue;
        const double x2 = zx * zx, y2 = zy * zy, r2 = x2 + y2, ir2 = 1.0 / r2;
        const double u = r2 * (side == 0 ? w.g_hi : w.g_lo), iu = 4.0 * ct * ir2;
        double e, F0, F1, F2;
        f_funcs<double>(u, iu, e, F0, F1, F2);
        const double E1 = e1x<double>(u, iu);
        const double pre = (side == 0 ? 1.0 : -1.0) * q * k.i4pk, nn = 2.0 * F0 * ir2;
        acc[0] -= pre * k.eta * (nn * x2 + E1 - F0);
        acc[1] -= pre * k.eta * (nn * y2 + E1 - F0);
        acc[2] -= pre * k.eta * (nn * zx * zy);
        acc[3] += pre * E1;
    }
}

// Dense product with exact element integrals, all in FP64 (DDM_MODE_DENSE |
// DDM_MODE_PRECISE): FP64 end points and unknowns in caller order; the DD
// part of every pair as its dislocation pair (the exact element integral at
// any distance), the fluid source by the 8-point Gauss-Legendre rule; the
// own element comes from the cached closed-form blocks (k_prep).  The FMM and
// the FP32 dense path carry FP32 geometry and pair arithmetic; this is the
// operator that escalated GMRES residuals of small problems use.  One thread
// per target, sources tiled through shared memory, blockIdx.y a source chunk.
constexpr int DX_T = 128;
__global__ void __launch_bounds__(DX_T) k_dense_exact(KConst<double> kd, Win<double> wd, const double *xy,
                                                      const double *x, int64_t N, int64_t chunk, double scale,
                                                      double *y) {
    __shared__ double sx0[DX_T], sy0[DX_T], sx1[DX_T], sy1[DX_T], sDx[DX_T], sDy[DX_T], sq[DX_T];
    const int64_t ti = blockIdx.x * (int64_t)DX_T + threadIdx.x;
    const bool act = ti < N;
    double mx = 0.0, my = 0.0, tx = 1.0, ty = 0.0;
    if (act) {
        const double ax = xy[ti], ay = xy[N + ti], bx = xy[2 * N + ti], by = xy[3 * N + ti];
        const double L = hypot(bx - ax, by - ay);
        mx = 0.5 * (ax + bx);
        my = 0.5 * (ay + by);
        tx = (bx - ax) / L;
        ty = (by - ay) / L;
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t s0 = blockIdx.y * chunk, s1 = s0 + chunk < N ? s0 + chunk : N;
    for (int64_t sb = s0; sb < s1; sb += DX_T) {
        __syncthreads();
        const int64_t sj = sb + threadIdx.x;
        if (sj < s1) {
            const double ax = xy[sj], ay = xy[N + sj], bx = xy[2 * N + sj], by = xy[3 * N + sj];
            const double L = hypot(bx - ax, by - ay), ux = (bx - ax) / L, uy = (by - ay) / L;
            const double Ds = x[sj], Dn = x[N + sj];
            sx0[threadIdx.x] = ax;
            sy0[threadIdx.x] = ay;
            sx1[threadIdx.x] = bx;
            sy1[threadIdx.x] = by;
            sDx[threadIdx.x] = Ds * ux - Dn * uy;          // D = Ds t + Dn n, n = (-t_y, t_x)
            sDy[threadIdx.x] = Ds * uy + Dn * ux;
            sq[threadIdx.x] = x[2 * N + sj];
        }
        __syncthreads();
        const int cnt = (int)(s1 - sb < DX_T ? s1 - sb : DX_T);
        if (act) {
            const double d4ct = 4.0 * (wd.ct_hi - wd.ct_lo);
            const double ce = wd.elastic ? kd.Cu : 0.0, pc = wd.elastic ? kd.pS : 0.0;
            const double fa0 = kd.a6 * d4ct, fq0 = -kd.qe * d4ct;
            for (int j = 0; j < cnt; ++j) {
                if (sb + j == ti) continue;
                {
                    // u > Big along the whole element: the exact integral of the
                    // rational large-u kernel (FP64: the remainders are below e^-70)
                    const double cx = 0.5 * (sx0[j] + sx1[j]), cy = 0.5 * (sy0[j] + sy1[j]);
                    const double hx = 0.5 * (sx1[j] - sx0[j]), hy = 0.5 * (sy1[j] - sy0[j]);   // a t
                    const double zx = mx - cx, zy = my - cy, a2 = hx * hx + hy * hy, a = sqrt(a2);
                    const double rb = a + wd.rbig;
                    if (zx * zx + zy * zy > rb * rb) {
                        const double nx = -hy / a, ny = hx / a;
                        const double pxx = sDx[j] * nx, pyy = sDy[j] * ny;
                        elem_bigu<double>(zx, zy, hx * hx - hy * hy, 2.0 * hx * hy, a2, 2.0 * a, pxx - pyy,
                                          sDx[j] * ny + sDy[j] * nx, pxx + pyy, sq[j], ce, pc, fa0, fq0, acc);
                        continue;
                    }
                }
                disl_field<double>(kd, mx - sx0[j], my - sy0[j], sDx[j], sDy[j], wd, 1.0, acc);    // start point
                disl_field<double>(kd, mx - sx1[j], my - sy1[j], sDx[j], sDy[j], wd, -1.0, acc);   // end point
                const double q = sq[j];
                if (q != 0.0) {
                    const double cx = 0.5 * (sx0[j] + sx1[j]), cy = 0.5 * (sy0[j] + sy1[j]);
                    const double hx = 0.5 * (sx1[j] - sx0[j]), hy = 0.5 * (sy1[j] - sy0[j]);   // a t
                    const double a = hypot(hx, hy);
#pragma unroll 1
                    for (int g = 0; g < 8; ++g)
                        q_point_d(kd, mx - cx - c_gl.x8[g] * hx, my - cy - c_gl.x8[g] * hy, c_gl.w8[g] * a * q, wd,
                                  acc);
                }
            }
        }
    }
    if (act) {
        double ss, sn;
        to_local<double>(tx, ty, acc, ss, sn);
        atomicAdd(&y[ti], scale * ss);
        atomicAdd(&y[N + ti], scale * sn);
        atomicAdd(&y[2 * N + ti], scale * acc[3]);
    }
}

}  // namespace

// ------------------------------------------------------------------- host
// The Gauss / Chebyshev tables live in __constant__ memory, which is global
// to the device: the last uploaded (n_cheb, quad_near) is tracked process
// wide, and contexts that use different values on one device must not run
// concurrently.
static std::mutex g_tab_mu;
static bool g_tab_done[64];
ddm_status upload_tables(ddm_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    int dv = ctx->device & 63;
    if (g_tab_done[dv]) return DDM_OK;
    GLTab h;
    memset(&h, 0, sizeof(h));
    double x[MAXGL], wt[MAXGL];
    for (int m = 1; m <= MAXGL; ++m) {
        gauss_legendre(m, x, wt);
        for (int i = 0; i < m; ++i) { h.xn[m][i] = (float)x[i]; h.wn[m][i] = (float)wt[i]; }
    }
    for (int n = 2; n <= DDM_MAX_CHEB; n += 2) {
        int o = n / 2 - 1;
        gauss_legendre(n, x, wt);
        for (int i = 0; i < n; ++i) { h.xc[o][i] = (float)x[i]; h.wc[o][i] = (float)wt[i]; }
        for (int j = 0; j < n; ++j) {
            double th = (2 * j + 1) * M_PI / (2.0 * n);
            h.cheb[o][j] = (float)cos(th);
            h.bw[o][j] = (float)(((j & 1) ? -1.0 : 1.0) * sin(th));
        }
    }
    gauss_legendre(8, h.x8, h.w8);
    DDM_CUDA_TRY(ctx, cudaMemcpyToSymbolAsync(c_gl, &h, sizeof(h), 0, cudaMemcpyHostToDevice, ctx->stream));
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    g_tab_done[dv] = true;
    return DDM_OK;
}

ddm_status ensure_workspace(ddm_ctx *ctx, ddm_tree *t) {
    int n = t->prm.n_cheb;
    if (t->ncheb_alloc == n && t->W) return DDM_OK;
    dfree(t->W, t->stream);
    dfree(t->Fl, t->stream);
    t->W = t->Fl = nullptr;
    size_t sz = (size_t)t->n_cells * 4 * n * n * sizeof(float);
    if (!t->far4 && dalloc(&t->far4, (size_t)t->n * sizeof(float4), t->stream) != cudaSuccess)
        return ctx_fail(ctx, DDM_ENOMEM, "FMM workspace allocation failed");
    if (dalloc(&t->W, sz, t->stream) != cudaSuccess || dalloc(&t->Fl, sz, t->stream) != cudaSuccess)
        return ctx_fail(ctx, DDM_ENOMEM, "FMM workspace allocation failed");
    t->ncheb_alloc = n;
    return DDM_OK;
}

template <class T>
static Win<T> make_win(const ddm_ctx *ctx, double lo, double hi) {
    Win<T> w;
    double c = ctx->kd.c;
    w.ct_hi = (T)(c * hi);
    w.ct_lo = (T)(lo > 0.0 ? c * lo : 0.0);
    w.g_hi = (T)(1.0 / (4.0 * c * hi));
    w.g_lo = (T)(lo > 0.0 ? 1.0 / (4.0 * c * lo) : 0.0);
    w.elastic = lo > 0.0 ? 0 : 1;
    w.rbig = (T)std::sqrt((double)Big<T>::U * 4.0 * c * hi);
    return w;
}

// own-element 3x3 blocks of the time window (lo, hi), from the tree's LRU
// window cache (computed on a miss, FP64 closed form, caller order)
ddm_status window_self_blocks(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s, const double **out) {
    const unsigned long long now = ++t->win_clock;
    int slot = -1;
    for (int k = 0; k < ddm_tree::WIN_CACHE; ++k)
        if (t->win_blk[k] && t->win_lo[k] == lo && t->win_hi[k] == hi) slot = k;
    if (slot < 0) {
        prof_begin(ctx, 1);
        slot = 0;                                  // an empty slot, else the least recently used
        for (int k = 0; k < ddm_tree::WIN_CACHE; ++k) {
            if (!t->win_blk[k]) { slot = k; break; }
            if (t->win_use[k] < t->win_use[slot]) slot = k;
        }
        const int64_t N = t->n;
        if (!t->win_blk[slot]) DDM_CUDA_TRY(ctx, dalloc(&t->win_blk[slot], 9 * N * sizeof(double), t->stream));
        k_self_blocks<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ctx->kd, make_win<double>(ctx, lo, hi), t->xy_caller,
                                                                  N, t->win_blk[slot]);
        DDM_CUDA_TRY(ctx, cudaGetLastError());
        t->win_lo[slot] = lo;
        t->win_hi[slot] = hi;
        prof_end(ctx, 1, 1);
    }
    t->win_use[slot] = now;
    *out = t->win_blk[slot];
    return DDM_OK;
}

// M2L operator set of window (lo, hi) for tree t from the tree's LRU cache,
// built on stream s when missing (one (4n^2)^2 matrix per (level, offset))
ddm_status window_ops(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s, const float **out) {
    const int n = t->prm.n_cheb, n2 = n * n, L = t->depth;
    const int nk = t->n_keys;
    const size_t opsz = (size_t)nk * 16 * n2 * n2;
    const unsigned long long now = t->win_clock;
    if (t->ops_n != n) {                       // new order: drop the cached sets
        for (int k = 0; k < ddm_tree::WIN_CACHE; ++k) {
            dfree(t->ops_set[k], t->stream);
            t->ops_set[k] = nullptr;
        }
        t->ops_n = n;
        // up to 4 GB of operator sets (at least one)
        t->ops_cap = (int)std::max<size_t>(1, std::min<size_t>(ddm_tree::WIN_CACHE, ((size_t)4 << 30) /
                                                               std::max<size_t>(1, opsz * sizeof(float))));
    }
    int os = -1;
    for (int k = 0; k < t->ops_cap; ++k)
        if (t->ops_set[k] && t->ops_lo[k] == lo && t->ops_hi[k] == hi) os = k;
    if (os >= 0) t->ops_use[os] = now;
    if (os < 0) {
        os = 0;
        for (int k = 0; k < t->ops_cap; ++k) {
            if (!t->ops_set[k]) { os = k; break; }
            if (t->ops_use[k] < t->ops_use[os]) os = k;
        }
        t->ops_use[os] = now;
        if (!t->ops_set[os]) DDM_CUDA_TRY(ctx, dalloc(&t->ops_set[os], opsz * sizeof(float), t->stream));
        prof_begin(ctx, 3);
        dim3 g((unsigned)((n2 * n2 + 127) / 128), (unsigned)nk);
        k_m2l_ops<<<g, 128, 0, s>>>(ctx->kf, make_win<float>(ctx, lo, hi), L, t->h0, n, t->mk_off, t->ops_set[os]);
        t->ops_lo[os] = lo;
        t->ops_hi[os] = hi;
        t->ops_cnt[os] = 0;
        prof_end(ctx, 3, 1);
    }
    *out = t->ops_set[os];
    return DDM_OK;
}

// Whether the M2L of window (lo, hi) on tree t takes the compressed
// operators: never (mode 0), whenever the order has a rank (mode 1), or
// (mode 2, the default) for orders n >= 10 once the window's full operators
// have served SVD_AUTO_USES products, so that only a window that keeps being
// applied (the operator of repeated solves at one time step) pays for the
// set-up.  A stream in capture never starts a set-up; it takes what is cached.
bool want_svd(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s) {
    const int n = t->prm.n_cheb;
    const int k = svd_rank(ctx, n);
    if (k <= 0 || ctx->m2l_compress == 0) return false;
    if (t->svd_k == k)
        for (int q = 0; q < ddm_tree::WIN_CACHE; ++q)
            if (t->svd_set[q] && t->svd_lo[q] == lo && t->svd_hi[q] == hi) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    if (ctx->m2l_compress == 1) return true;
    if (n < 10 || t->ops_n != n) return false;
    for (int k = 0; k < t->ops_cap; ++k)
        if (t->ops_set[k] && t->ops_lo[k] == lo && t->ops_hi[k] == hi) return ++t->ops_cnt[k] > SVD_AUTO_USES;
    return false;
}

// Compressed M2L of window (lo, hi) for tree t: bases and cores from the
// tree's LRU cache (built from the window's full operators when missing),
// the per-level cell lists of the pre- and post-stages and the k-per-cell
// work arrays (once per tree).
ddm_status window_svd(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s, const float **pre,
                      const float **post, const float **core) {
    const int n = t->prm.n_cheb, ld = 4 * n * n, k = svd_rank(ctx, n), L = t->depth;
    if (t->svd_k != k) {                 // another rank: drop the cached sets and work arrays
        if (t->svd_k) DDM_CUDA_TRY(ctx, cudaDeviceSynchronize());   // products in flight may read them
        for (int q = 0; q < ddm_tree::WIN_CACHE; ++q) {
            dfree(t->svd_set[q], t->stream);
            t->svd_set[q] = nullptr;
        }
        dfree(t->Wc, t->stream);
        dfree(t->Gc, t->stream);
        t->Wc = t->Gc = nullptr;
        t->svd_k = k;
    }
    if (!t->Wc) {
        DDM_CUDA_TRY(ctx, dalloc(&t->Wc, (size_t)t->n_cells * k * sizeof(float), t->stream));
        DDM_CUDA_TRY(ctx, dalloc(&t->Gc, (size_t)t->n_cells * k * sizeof(float), t->stream));
    }
    if (!t->lv_off) {
        std::vector<int32_t> off(L + 2, 0);
        std::vector<int2> pairs, work;
        for (int l = 0; l <= L; ++l) {
            off[l] = (int32_t)pairs.size();
            if (l < 2) continue;
            for (int64_t c = t->lvl_off[l]; c < t->lvl_off[l + 1]; ++c) pairs.push_back(make_int2((int)c, (int)c));
            for (int32_t p = off[l]; p < (int32_t)pairs.size(); p += 64) work.push_back(make_int2(l, p));
        }
        off[L + 1] = (int32_t)pairs.size();
        t->n_lv_work = (int)work.size();
        DDM_CUDA_TRY(ctx, dalloc(&t->lv_off, off.size() * sizeof(int32_t), t->stream));
        DDM_CUDA_TRY(ctx, dalloc(&t->lv_pair, std::max<size_t>(1, pairs.size()) * sizeof(int2), t->stream));
        DDM_CUDA_TRY(ctx, dalloc(&t->lv_work, std::max<size_t>(1, work.size()) * sizeof(int2), t->stream));
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(t->lv_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                          t->stream));
        if (!pairs.empty())
            DDM_CUDA_TRY(ctx, cudaMemcpyAsync(t->lv_pair, pairs.data(), pairs.size() * sizeof(int2),
                                              cudaMemcpyHostToDevice, t->stream));
        if (!work.empty())
            DDM_CUDA_TRY(ctx, cudaMemcpyAsync(t->lv_work, work.data(), work.size() * sizeof(int2),
                                              cudaMemcpyHostToDevice, t->stream));
        DDM_CUDA_TRY(ctx, cudaStreamSynchronize(t->stream));   // host lists go out of scope
    }
    const size_t npre = (size_t)(L + 1) * k * ld, ncore = (size_t)t->n_keys * k * k;
    const unsigned long long now = t->win_clock;
    int os = -1;
    for (int q = 0; q < ddm_tree::WIN_CACHE; ++q)
        if (t->svd_set[q] && t->svd_lo[q] == lo && t->svd_hi[q] == hi) os = q;
    if (os >= 0) t->svd_use[os] = now;
    if (os < 0) {
        os = 0;
        for (int q = 0; q < ddm_tree::WIN_CACHE; ++q) {
            if (!t->svd_set[q]) { os = q; break; }
            if (t->svd_use[q] < t->svd_use[os]) os = q;
        }
        t->svd_use[os] = now;
        if (!t->svd_set[os]) DDM_CUDA_TRY(ctx, dalloc(&t->svd_set[os], (2 * npre + ncore) * sizeof(float), t->stream));
        const float *ops = nullptr;
        ddm_status st = window_ops(ctx, t, lo, hi, s, &ops);
        if (st) return st;
        float *b = t->svd_set[os];
        if ((st = svd_build(ctx, t, ops, k, s, b, b + npre, b + 2 * npre))) return st;
        t->svd_lo[os] = lo;
        t->svd_hi[os] = hi;
    }
    *pre = t->svd_set[os];
    *post = t->svd_set[os] + npre;
    *core = t->svd_set[os] + 2 * npre;
    return DDM_OK;
}

ddm_status op_apply(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, const double *x, double *y, int mode,
                    int accumulate, double scale, cudaStream_t stream_override) {
    const bool precise = (mode & DDM_MODE_PRECISE) != 0;
    mode &= ~DDM_MODE_PRECISE;
    if (!(hi > lo) || lo < 0.0) return ctx_fail(ctx, DDM_EINVAL, "matvec: need 0 <= tau_lo < tau_hi");
    ddm_status st = upload_tables(ctx);
    if (st) return st;
    st = ensure_workspace(ctx, t);
    if (st) return st;
    cudaStream_t s = stream_override ? stream_override : ctx->stream;
    int64_t N = t->n;
    int n = t->prm.n_cheb, n2 = n * n;
    const int nq = t->prm.quad_near;
    const int TB = 256;
    KConst<float> kf = ctx->kf;
    Win<float> wf = make_win<float>(ctx, lo, hi);
    Win<double> wd = make_win<double>(ctx, lo, hi);
    // own-element blocks of this time window (FP64 closed form), cached
    const double *blk = nullptr;
    st = window_self_blocks(ctx, t, lo, hi, s, &blk);
    if (st) return st;
    const int overwrite = accumulate ? 0 : 1;
    const int L = t->depth;                   // deepest level
    const int64_t nleaf = t->n_leaf;
    const float h0f = (float)t->h0;           // leaf half-widths h0 2^-level, exact in FP32
    int use_far = mode != DDM_MODE_DENSE && L >= 2;
    {
        // charges; for the far field also zero the weights and local
        // expansions of the cells on levels 2 .. L (the upward pass and the
        // M2L add into them)
        const int64_t z0 = use_far ? t->lvl_off[2] : 0, z1 = use_far ? t->lvl_off[L + 1] : 0;
        const int64_t nz = (z1 - z0) * 4 * (int64_t)n2;
        prof_begin(ctx, 0);
        k_prep<<<(unsigned)std::max<int64_t>((N + TB - 1) / TB, 1), TB, 0, s>>>(
            x, t->perm, t->g_frame, blk, N, scale, overwrite, t->chg, y, t->W + z0 * 4 * n2, t->Fl + z0 * 4 * n2, nz);
        prof_end(ctx, 0, 1);
    }
    if (mode == DDM_MODE_DENSE && precise) {
        const int64_t tiles = (N + DX_T - 1) / DX_T;
        int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + tiles - 1) / tiles, tiles));
        int64_t chunk = ((N + chunks - 1) / chunks + DX_T - 1) / DX_T * DX_T;
        chunks = (N + chunk - 1) / chunk;
        prof_begin(ctx, 7);
        k_dense_exact<<<dim3((unsigned)tiles, (unsigned)chunks), DX_T, 0, s>>>(ctx->kd, wd, t->xy_caller, x, N, chunk,
                                                                               scale, y);
        prof_end(ctx, 7, 1);
        DDM_CUDA_TRY(ctx, cudaGetLastError());
        return DDM_OK;
    }
    if (mode == DDM_MODE_DENSE) {
        int64_t tiles = (N + DN_T - 1) / DN_T;
        int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + tiles - 1) / tiles, (N + DN_T - 1) / DN_T));
        int64_t chunk = ((N + chunks - 1) / chunks + DN_T - 1) / DN_T * DN_T;
        chunks = (N + chunk - 1) / chunk;
        prof_begin(ctx, 7);
        auto kdn = k_dense<false>;          // precise dense products take k_dense_exact above
        kdn<<<dim3((unsigned)tiles, (unsigned)chunks), DN_T, 0, s>>>(kf, ctx->kd, wf, wd, nq, t->g_loc, t->g_grid,
                                                                     t->g16, t->g_frame, t->chg, t->perm, N, chunk,
                                                                     scale, y);
        prof_end(ctx, 7, 1);
        DDM_CUDA_TRY(ctx, cudaGetLastError());
        return DDM_OK;
    }
    // The near field needs only the charges: unless profiling or capturing
    // (stream given), it runs on the context stream while the far field
    // (upward pass, M2L, L2L) runs on the auxiliary stream, and L2P follows
    // the join.
    const bool overlap = use_far && stream_override == nullptr && !ctx->prof.on;
    cudaStream_t fs = overlap ? ctx->aux : s;
    if (use_far) {
        if (overlap) {
            DDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, s));
            DDM_CUDA_TRY(ctx, cudaStreamWaitEvent(fs, ctx->ev_fork, 0));
        }
        // upward pass: P2M and M2M in one launch
        prof_begin(ctx, 2);
#define DDM_UP(NN)                                                                                          \
    k_up<NN><<<(unsigned)t->n_up_items, UP_T, 0, fs>>>(t->up_items, t->leaf_at, h0f, t->cell_ix, t->cell_iy,       \
                                                       t->cell_parent, t->g_rel, t->g_frame, t->chg, t->W,           \
                                                       ctx->cheb_Tn[NN / 2 - 1])
        DDM_CHEB_SWITCH(n, DDM_UP);
#undef DDM_UP
        prof_end(ctx, 2, 1);
        // M2L on every level >= 2: operators of this window, then one GEMM launch
        // (compressed: three)
        const int kr = want_svd(ctx, t, lo, hi, fs) ? svd_rank(ctx, n) : 0;
        const float *ops = nullptr, *spre = nullptr, *spost = nullptr, *score = nullptr;
        if (kr > 0) {
            if ((st = window_svd(ctx, t, lo, hi, fs, &spre, &spost, &score))) return st;
        } else if ((st = window_ops(ctx, t, lo, hi, fs, &ops))) {
            return st;
        }
        prof_begin(ctx, 4);
        // (the local expansions of every cell at levels >= 2 were zeroed by k_up)
        if (t->n_work > 0 && kr > 0) {
            static bool attr_g[64] = {false};
            if (!attr_g[ctx->device & 63]) {
                DDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       tc::SMEM_BYTES));
                attr_g[ctx->device & 63] = true;
            }
            // W' = (V^T D_in^-1) W per cell, G' = C W' per pair, F += (D_out^-1 U) G' per cell.
            // The per-cell stages have few column tiles (64 cells each): their
            // K range is split over gridDim.z blocks whose sums meet in the
            // output atomics
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(t->Wc, 0, (size_t)t->n_cells * kr * sizeof(float), fs));
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(t->Gc, 0, (size_t)t->n_cells * kr * sizeof(float), fs));
            const int ld = 4 * n2;
            // (a split that leaves every block at least one K chunk: the
            // accumulator of a block without one would hold no product)
            auto ksplit = [](int Kd, int want) {
                const int nkt = (Kd + tc::BK - 1) / tc::BK, per = (nkt + want - 1) / want;
                return (nkt + per - 1) / per;
            };
            const int kpre = ksplit(ld, std::max(1, std::min(8, (ld + tc::BK - 1) / tc::BK / 2)));
            const int kpost = ksplit(kr, 4);
            k_tc_group<<<dim3((unsigned)t->n_lv_work, (unsigned)((kr + tc::BM - 1) / tc::BM), (unsigned)kpre),
                         tc::THREADS, tc::SMEM_BYTES, fs>>>(t->lv_work, t->lv_off, t->lv_pair, kr, ld, spre, t->W,
                                                            t->Wc, ctx->d_err);
            k_tc_group<<<dim3((unsigned)t->n_work, (unsigned)((kr + tc::BM - 1) / tc::BM)), tc::THREADS,
                         tc::SMEM_BYTES, fs>>>(t->mk_work, t->mk_off, t->mk_pair, kr, kr, score, t->Wc, t->Gc,
                                               ctx->d_err);
            k_tc_group<<<dim3((unsigned)t->n_lv_work, (unsigned)((ld + tc::BM - 1) / tc::BM), (unsigned)kpost),
                         tc::THREADS, tc::SMEM_BYTES, fs>>>(t->lv_work, t->lv_off, t->lv_pair, ld, kr, spost, t->Gc,
                                                            t->Fl, ctx->d_err);
        } else if (t->n_work > 0) {
            static bool attr[64] = {false};
            if (!attr[ctx->device & 63]) {
                DDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       tc::SMEM_BYTES));
                attr[ctx->device & 63] = true;
            }
            dim3 g((unsigned)t->n_work, (unsigned)((4 * n2 + tc::BM - 1) / tc::BM),
                   (unsigned)std::min(tc::KSPLIT, (4 * n2 + tc::BK - 1) / tc::BK));
            k_m2l_tc<<<g, tc::THREADS, tc::SMEM_BYTES, fs>>>(t->mk_work, t->mk_off, t->mk_pair, n, ops, t->W,
                                                            t->Fl, ctx->d_err);
        }
        prof_end(ctx, 4, (t->n_work > 0 && kr > 0) ? 3 : 1);
        // downward pass: L2L chains to the leaves and L2P at their targets, one launch
        prof_begin(ctx, 5);
#define DDM_DOWN(NN)                                                                                        \
    k_down<NN><<<(unsigned)nleaf, L2L_T, 0, fs>>>(t->leaf_at, h0f, t->cell_ix, t->cell_iy, t->cell_parent,           \
                                                  ctx->cheb_Tn[n / 2 - 1], t->Fl, t->cell_start, t->cell_end, t->g_rel, \
                                                  t->far4, t->g_frame, t->perm, N, scale, precise ? nullptr : y)
        DDM_CHEB_SWITCH(n, DDM_DOWN);
#undef DDM_DOWN
        prof_end(ctx, 5, 1);
    }
    if (overlap) DDM_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_join, fs));
    prof_begin(ctx, 6);
    if (precise)
        k_near<true><<<(unsigned)((N + NEAR_W - 1) / NEAR_W), NEAR_T, 0, s>>>(
            kf, ctx->kd, wf, wd, t->nb_off, t->nb_tab, t->elem_leaf, t->g_rel, t->g_loc, t->g_grid, t->g16,
            t->g_frame, t->chg, t->perm, t->leaf_at, h0f, n, nq, t->Fl, 0, N, scale, y);
    else
        (lo > 0.0 ? k_near2<true> : k_near2<false>)<<<(unsigned)((t->n_items + NEAR_W - 1) / NEAR_W), NEAR_T, 0, s>>>(
            kf, wf, t->nb_off, t->nb_tab, t->elem_leaf, t->g_loc, t->g_grid, t->g_frame, t->chg, t->perm, t->g16, nq,
            t->near_items, t->n_items, N, scale, y);
    prof_end(ctx, 6, 1);
    if (use_far) {
        if (overlap) DDM_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
        // (plain products: k_down added the far field into y itself; the
        // precise near kernel writes y plainly, so its far field follows here)
        if (precise) k_far_add<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(t->far4, t->g_frame, t->perm, N, scale, y);
    }
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

// ---------------------------------------------------------------------------
// Many problems' FMM products in one launch per stage.
//
// A batch of independent problems (trees of the same Chebyshev order) is
// advanced stage by stage: charges and own elements, upward pass, M2L,
// downward pass, near field, far-field add.  Each stage is one launch over a
// work list of (problem, local unit) entries built once on the host; the
// per-problem arrays are reached through a descriptor table.  The upward and
// downward passes, the near field and the element stages run persistent
// grids (a multiple of the SM count) that stride over the list, the M2L one
// CTA per (problem, column tile) as in a single product.  Small problems thus
// share the device with large ones instead of running one narrow grid each.
// ---------------------------------------------------------------------------
namespace {
struct BDesc {
    const double *x;
    double *y;
    const int64_t *perm;
    const float4 *g_frame, *g_rel, *g_loc;
    const float2 *g_grid;
    const double *blk;
    float4 *chg;
    float *W, *Fl;
    float4 *far4;
    const int32_t *cstart, *cend, *cix, *ciy, *parent;
    const int32_t *nb_off;
    const int4 *nb_tab;
    const int32_t *elem_leaf;
    const int2 *near_items;
    const int2 *mk_work;
    const int32_t *mk_off;
    const int2 *mk_pair;
    const float *ops;
    const int2 *leaf_at;
    const int4 *up_items;
    int64_t n, zoff;
    int L, nq;
    float h0, g16;
};
constexpr int BE_T = 256, BE_CHUNK = 1024;
// items (p, kind, a, b): kind 0 prepares elements [a, b), kind 1 zeroes the
// expansions of the cells of levels >= 2, floats [zoff + a, zoff + b)
// act (may be null): per-problem flags, items of problems whose flag is 0
// are skipped (the same work lists serve every subset of the problems)
__global__ void __launch_bounds__(BE_T) k_prep_b(const BDesc *D, const int4 *items, int nitems, double scale,
                                                 int overwrite, const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        if (act && !act[w.x]) continue;
        const BDesc &d = D[w.x];
        if (w.y == 0) {
            for (int64_t i = w.z + threadIdx.x; i < w.w; i += BE_T)
                prep_elem(i, d.x, d.perm, d.g_frame, d.blk, d.n, scale, overwrite, d.chg, d.y);
        } else {
            for (int64_t z = w.z + threadIdx.x; z < w.w; z += BE_T) {
                d.W[d.zoff + z] = 0.f;
                d.Fl[d.zoff + z] = 0.f;
            }
        }
    }
}
template <int N>
__global__ void __launch_bounds__(UP_T) k_up_b(const BDesc *D, const int2 *items, int nitems, const float *T,
                                               const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        if (act && !act[w.x]) continue;      // uniform over the block
        const BDesc &d = D[w.x];
        up_body<N>(d.up_items, d.leaf_at, d.h0, d.cix, d.ciy, d.parent, d.g_rel, d.g_frame, d.chg, d.W, T, w.y);
        __syncthreads();                      // shared staging is reused by the next item
    }
}
template <int N>
__global__ void __launch_bounds__(L2L_T) k_down_b(const BDesc *D, const int2 *items, int nitems, const float *T,
                                                  const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        if (act && !act[w.x]) continue;
        const BDesc &d = D[w.x];
        down_body<N>(d.leaf_at, d.h0, d.cix, d.ciy, d.parent, T, d.Fl, d.cstart, d.cend, d.g_rel, d.far4, nullptr,
                     nullptr, 0, 0.0, nullptr, w.y);
        __syncthreads();
    }
}
__global__ void __launch_bounds__(tc::THREADS) k_m2l_tc_b(const BDesc *D, const int2 *items, int n, int *err,
                                                          const int *act) {
    const int2 w = items[blockIdx.x];
    if (act && !act[w.x]) return;            // whole CTA, before any tensor-memory allocation
    const BDesc &d = D[w.x];
    m2l_body(d.mk_work, d.mk_off, d.mk_pair, n, d.ops, d.W, d.Fl, err, w.y);
}
template <bool TWO>
__global__ void __launch_bounds__(NEAR_T, 4) k_near2_b(KConst<float> k, Win<float> win, const BDesc *D,
                                                       const int2 *items, int64_t nitems, double scale,
                                                       const int *act) {
    // one item per warp (a loop over items would cost the body registers)
    const int64_t g = (int64_t)blockIdx.x * NEAR_W + (threadIdx.x >> 5);
    if (g >= nitems) return;
    const int2 w = items[g];
    if (act && !act[w.x]) return;
    const BDesc &d = D[w.x];
    near2_body<TWO>(k, win, d.nb_off, d.nb_tab, d.elem_leaf, d.g_loc, d.g_grid, d.g_frame, d.chg, d.perm, d.g16,
                    d.nq, d.near_items, d.n, scale, d.y, w.y);
}
// items (p, 0, a, b): far field of elements [a, b) into y
__global__ void __launch_bounds__(BE_T) k_far_add_b(const BDesc *D, const int4 *items, int nitems, double scale,
                                                    const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        if (act && !act[w.x]) continue;
        const BDesc &d = D[w.x];
        for (int64_t ti = w.z + threadIdx.x; ti < w.w; ti += BE_T) {
            const float4 g4 = d.far4[ti], f = d.g_frame[ti];
            const float g[4] = {g4.x, g4.y, g4.z, g4.w};
            float ss, sn;
            to_local<float>(f.x, f.y, g, ss, sn);
            const int64_t e = d.perm[ti];
            d.y[e] += scale * (double)ss;
            d.y[d.n + e] += scale * (double)sn;
            d.y[2 * d.n + e] += scale * (double)g4.w;
        }
    }
}
}  // namespace

struct BatchFmm {
    int n = 0, np = 0, nsm = 152;
    double lo = 0, hi = 0;
    BDesc *desc = nullptr;
    int4 *prep = nullptr, *far = nullptr;
    int2 *leaf = nullptr, *upit = nullptr, *m2l = nullptr, *near = nullptr;
    int n_prep = 0, n_far = 0, n_leaf = 0, n_up = 0, n_m2l = 0;
    int64_t n_near = 0;
    long long launches = 0;
    const int *act = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

void bfmm_free(BatchFmm *b, cudaStream_t s) {
    if (!b) return;
    void *ps[] = {b->desc, b->prep, b->far, b->leaf, b->upit, b->m2l, b->near};
    for (void *p : ps) dfree(p, s);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
}

ddm_status bfmm_build(ddm_ctx *ctx, ddm_tree *const *trees, int np, const int *idx, int nidx, double lo, double hi,
                      const double *const *xs, double *const *ys, const int *act, cudaStream_t s, BatchFmm **out) {
    *out = nullptr;
    if (np <= 0 || nidx <= 0) return ctx_fail(ctx, DDM_EINVAL, "batched product: no problems");
    const int n = trees[idx[0]]->prm.n_cheb, n2 = n * n;
    ddm_status st = upload_tables(ctx);
    if (st) return st;
    std::vector<BDesc> hd(np);
    std::memset(hd.data(), 0, hd.size() * sizeof(BDesc));
    std::vector<int4> hprep, hfar;
    std::vector<int2> hleaf, hup, hm2l, hnear;
    for (int q = 0; q < nidx; ++q) {
        const int p = idx[q];
        ddm_tree *t = trees[p];
        if (t->prm.n_cheb != n) return ctx_fail(ctx, DDM_EINVAL, "batched product: trees of different orders");
        if ((st = ensure_workspace(ctx, t))) return st;
        const double *blk = nullptr;
        if ((st = window_self_blocks(ctx, t, lo, hi, s, &blk))) return st;
        const int L = t->depth;
        const bool far = L >= 2;
        const float *ops = nullptr;
        if (far && (st = window_ops(ctx, t, lo, hi, s, &ops))) return st;
        const int64_t nleaf = t->n_leaf;
        BDesc &d = hd[p];
        d.x = xs[p]; d.y = ys[p];
        d.perm = t->perm; d.g_frame = t->g_frame; d.g_rel = t->g_rel; d.blk = blk;
        d.g_loc = t->g_loc; d.g_grid = t->g_grid; d.g16 = t->g16;
        d.chg = t->chg; d.W = t->W; d.Fl = t->Fl; d.far4 = t->far4;
        d.cstart = t->cell_start; d.cend = t->cell_end; d.cix = t->cell_ix; d.ciy = t->cell_iy;
        d.parent = t->cell_parent;
        d.nb_off = t->nb_off; d.nb_tab = t->nb_tab; d.elem_leaf = t->elem_leaf; d.near_items = t->near_items;
        d.mk_work = t->mk_work; d.mk_off = t->mk_off; d.mk_pair = t->mk_pair; d.ops = ops;
        d.n = t->n; d.leaf_at = t->leaf_at; d.up_items = t->up_items; d.L = L; d.nq = t->prm.quad_near; d.h0 = (float)t->h0;
        d.zoff = far ? t->lvl_off[2] * 4 * n2 : 0;
        for (int64_t a = 0; a < t->n; a += BE_CHUNK) {
            const int b = (int)std::min<int64_t>(t->n, a + BE_CHUNK);
            hprep.push_back(make_int4(p, 0, (int)a, b));
            if (far) hfar.push_back(make_int4(p, 0, (int)a, b));
        }
        if (far) {
            const int64_t nz = (t->lvl_off[L + 1] - t->lvl_off[2]) * 4 * n2;
            for (int64_t a = 0; a < nz; a += 8 * BE_CHUNK)
                hprep.push_back(make_int4(p, 1, (int)a, (int)std::min<int64_t>(nz, a + 8 * BE_CHUNK)));
            for (int64_t l = 0; l < nleaf; ++l) hleaf.push_back(make_int2(p, (int)l));
            for (int64_t u = 0; u < t->n_up_items; ++u) hup.push_back(make_int2(p, (int)u));
            for (int w = 0; w < t->n_work; ++w) hm2l.push_back(make_int2(p, w));
        }
        for (int64_t i = 0; i < t->n_items; ++i) hnear.push_back(make_int2(p, (int)i));
    }
    {   // (outside any stream capture: the batch's launches may be captured later)
        static bool attr[64] = {false};
        if (!attr[ctx->device & 63]) {
            DDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_m2l_tc_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   tc::SMEM_BYTES));
            attr[ctx->device & 63] = true;
        }
    }
    BatchFmm *b = new BatchFmm();
    b->n = n; b->np = np; b->lo = lo; b->hi = hi; b->act = act;
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    b->n_prep = (int)hprep.size(); b->n_far = (int)hfar.size(); b->n_leaf = (int)hleaf.size();
    b->n_up = (int)hup.size();
    b->n_m2l = (int)hm2l.size(); b->n_near = (int64_t)hnear.size();
    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        if (dalloc(dst, bytes ? bytes : 16, s) != cudaSuccess) return false;
        return !bytes || cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    bool ok = up((void **)&b->desc, hd.data(), hd.size() * sizeof(BDesc)) &&
              up((void **)&b->prep, hprep.data(), hprep.size() * sizeof(int4)) &&
              up((void **)&b->far, hfar.data(), hfar.size() * sizeof(int4)) &&
              up((void **)&b->leaf, hleaf.data(), hleaf.size() * sizeof(int2)) &&
              up((void **)&b->upit, hup.data(), hup.size() * sizeof(int2)) &&
              up((void **)&b->m2l, hm2l.data(), hm2l.size() * sizeof(int2)) &&
              up((void **)&b->near, hnear.data(), hnear.size() * sizeof(int2)) &&
              cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess;       // host item lists go out of scope
    if (!ok) {
        bfmm_free(b, s);
        return ctx_fail(ctx, DDM_ENOMEM, "batched product: work list allocation failed");
    }
    *out = b;
    return DDM_OK;
}

// The stages of every problem's product y = [K(hi) - K(lo)] x (overwrite)
// on stream s, the far branch (upward pass, M2L, downward pass) forked to
// aux when given (aux = nullptr: all on s).
ddm_status bfmm_launch(ddm_ctx *ctx, BatchFmm *b, cudaStream_t s, cudaStream_t aux) {
    const int n = b->n;
    const int nsm = b->nsm;
    auto grid = [&](int64_t items, int per_sm) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)nsm * per_sm)); };
    long long launches = 0;
    k_prep_b<<<grid(b->n_prep, 8), BE_T, 0, s>>>(b->desc, b->prep, b->n_prep, 1.0, 1, b->act);
    ++launches;
    cudaStream_t fs = aux ? aux : s;
    if (b->n_leaf > 0) {
        if (aux) {
            DDM_CUDA_TRY(ctx, cudaEventRecord(b->ev_fork, s));
            DDM_CUDA_TRY(ctx, cudaStreamWaitEvent(fs, b->ev_fork, 0));
        }
#define DDM_UPB(NN) k_up_b<NN><<<grid(b->n_up, 4), UP_T, 0, fs>>>(b->desc, b->upit, b->n_up, ctx->cheb_Tn[NN / 2 - 1], b->act)
        DDM_CHEB_SWITCH(n, DDM_UPB);
#undef DDM_UPB
        if (b->n_m2l > 0) {
            dim3 g((unsigned)b->n_m2l, (unsigned)((4 * n * n + tc::BM - 1) / tc::BM), 1);
            k_m2l_tc_b<<<g, tc::THREADS, tc::SMEM_BYTES, fs>>>(b->desc, b->m2l, n, ctx->d_err, b->act);
            ++launches;
        }
#define DDM_DOWNB(NN) k_down_b<NN><<<grid(b->n_leaf, 8), L2L_T, 0, fs>>>(b->desc, b->leaf, b->n_leaf, ctx->cheb_Tn[NN / 2 - 1], b->act)
        DDM_CHEB_SWITCH(n, DDM_DOWNB);
#undef DDM_DOWNB
        launches += 2;
        if (aux) DDM_CUDA_TRY(ctx, cudaEventRecord(b->ev_join, fs));
    }
    if (b->n_near > 0) {
        auto kn = b->lo > 0.0 ? k_near2_b<true> : k_near2_b<false>;
        kn<<<(unsigned)((b->n_near + NEAR_W - 1) / NEAR_W), NEAR_T, 0, s>>>(
            ctx->kf, make_win<float>(ctx, b->lo, b->hi), b->desc, b->near, b->n_near, 1.0, b->act);
        ++launches;
    }
    if (b->n_leaf > 0) {
        if (aux) DDM_CUDA_TRY(ctx, cudaStreamWaitEvent(s, b->ev_join, 0));
        k_far_add_b<<<grid(b->n_far, 8), BE_T, 0, s>>>(b->desc, b->far, b->n_far, 1.0, b->act);
        ++launches;
    }
    prof_end(ctx, 6, (int)launches);
    b->launches = launches;
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free dense product.
//
// Some callers cannot allocate device memory at the point where they need a
// product: a real-time loop that forbids allocation after start-up, code
// running inside another framework's fixed memory budget, or code called
// while that framework holds its allocator.  ddm_matvec_dense_static serves
// them: it needs no tree, no workspace and no allocation.  Its only scratch
// (per element: FP64 midpoint, FP32 frame and DD charges) is this file-scope
// device array, sized for DDM_STATIC_MAX_ELEMENTS elements (48 B each,
// 3 MB), which every GPU that loads the library holds until the process
// exits.  All calls share the array, so calls whose work overlaps on the GPU
// race; each call rewrites the entries of its n elements before reading them,
// and nothing in the array needs to start at zero.  A one-word flag beside
// it, cleared by every call, marks invalid geometry.
// ---------------------------------------------------------------------------
namespace {
struct StaticElem {
    double2 mid;     // midpoint (FP64)
    float4 frame;    // tangent (x, y), half-length, unused
    float4 chg;      // global DD vector (x, y), fluid source, unused
};
static __device__ __align__(256) StaticElem g_static_scratch[DDM_STATIC_MAX_ELEMENTS];
// raised by the preparation kernel for an element of zero length or with a
// non-finite end point (cleared at the start of every call)
static __device__ int g_static_bad;

std::mutex g_static_mu;
StaticElem *g_static_ptr[256] = {nullptr};   // device address of the array, per device
int *g_static_bad_ptr[256] = {nullptr};      // device address of the flag, per device

__global__ void k_static_prep(const double *xy, const double *x, int64_t n, StaticElem *sc, int *bad) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double ax = xy[e], ay = xy[n + e], bx = xy[2 * n + e], by = xy[3 * n + e];
    double L = hypot(bx - ax, by - ay), tx = (bx - ax) / L, ty = (by - ay) / L;
    if (!(L > 0.0) || !isfinite(L) || !isfinite(ax) || !isfinite(ay)) *bad = 1;
    float Ds = (float)x[e], Dn = (float)x[n + e], Dq = (float)x[2 * n + e];
    float ftx = (float)tx, fty = (float)ty;
    StaticElem s;
    s.mid = make_double2(0.5 * (ax + bx), 0.5 * (ay + by));
    s.frame = make_float4(ftx, fty, (float)(0.5 * L), 0.f);
    s.chg = make_float4(Ds * ftx - Dn * fty, Ds * fty + Dn * ftx, Dq, 0.f);
    sc[e] = s;
}

// one thread per target, all sources through shared memory tiles; pair
// offsets from FP64 midpoints, own element in FP64 closed form
constexpr int ST_T = 128;
__global__ void __launch_bounds__(ST_T) k_static_dense(KConst<float> k, KConst<double> kd, Win<float> w,
                                                       Win<double> wd, int nq, const StaticElem *sc, const double *x,
                                                       int64_t n, double *y, const int *bad) {
    __shared__ StaticElem tile[ST_T];
    int64_t ti = blockIdx.x * (int64_t)ST_T + threadIdx.x;
    if (*bad) {          // invalid geometry: every output is NaN, nothing else is read
        if (ti < n) y[ti] = y[n + ti] = y[2 * n + ti] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    bool act = ti < n;
    StaticElem me = act ? sc[ti] : sc[0];
    double accd[4] = {0, 0, 0, 0};
    for (int64_t sb = 0; sb < n; sb += ST_T) {
        __syncthreads();
        if (sb + threadIdx.x < n) tile[threadIdx.x] = sc[sb + threadIdx.x];
        __syncthreads();
        int cnt = (int)(n - sb < ST_T ? n - sb : ST_T);
        if (act) {
            float acc[4] = {0, 0, 0, 0};
            for (int j = 0; j < cnt; ++j) {
                if (sb + j == ti) continue;
                const StaticElem &o = tile[j];
                float cx = (float)(o.mid.x - me.mid.x), cy = (float)(o.mid.y - me.mid.y);
                SrcTile st;
                st.x0 = cx - o.frame.z * o.frame.x; st.y0 = cy - o.frame.z * o.frame.y;
                st.x1 = cx + o.frame.z * o.frame.x; st.y1 = cy + o.frame.z * o.frame.y;
                st.Dx = o.chg.x; st.Dy = o.chg.y; st.q = o.chg.z; st.a = o.frame.z;
                st.tx = o.frame.x; st.ty = o.frame.y; st.idx = (int)(sb + j);
                pair_field<false>(k, kd, w, wd, nq, 0.f, 0.f, st, acc, accd);
            }
            for (int c = 0; c < 4; ++c) accd[c] += (double)acc[c];
        }
    }
    if (!act) return;
    double tx = (double)me.frame.x, ty = (double)me.frame.y, ss, sn;
    to_local<double>(tx, ty, accd, ss, sn);
    double o[3];
    self_field(kd, wd, (double)me.frame.z, tx, ty, x[ti], x[n + ti], x[2 * n + ti], o);
    y[ti] = ss + o[0];
    y[n + ti] = sn + o[1];
    y[2 * n + ti] = accd[3] + o[2];
}
}  // namespace

extern "C" ddm_status ddm_matvec_dense_static(ddm_ctx *ctx, const double *d_xy, int64_t n, double tau_lo,
                                              double tau_hi, const double *d_x, double *d_y) {
    if (!ctx || !d_xy || !d_x || !d_y)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: bad arguments");
    if (n <= 0 || n > DDM_STATIC_MAX_ELEMENTS)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: n must be in [1, " +
                                             std::to_string(DDM_STATIC_MAX_ELEMENTS) + "], got " + std::to_string(n));
    {   // d_y is written while d_x is still read: the 3n ranges must not overlap
        const uintptr_t xa = (uintptr_t)d_x, ya = (uintptr_t)d_y, len = (uintptr_t)(3 * n) * sizeof(double);
        if (xa < ya + len && ya < xa + len)
            return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: d_x and d_y overlap");
    }
    if (!(tau_hi > tau_lo) || tau_lo < 0.0)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: need 0 <= tau_lo < tau_hi");
    int dev = 0;
    DDM_CUDA_TRY(ctx, cudaGetDevice(&dev));
    if (dev != ctx->device)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: the context's device must be current");
    if (dev < 0 || dev >= 256) return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: device index out of range");
    StaticElem *sc = nullptr;
    int *bad = nullptr;
    {
        // set-up, once per device, with that device current: the host-side
        // names of the array and the flag are not device addresses; ask the
        // runtime for them
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *p = nullptr, *q = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_static_bad);
            if (e != cudaSuccess)
                return ctx_fail(ctx, DDM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_static_bad_ptr[dev] = (int *)q;
            g_static_ptr[dev] = (StaticElem *)p;
        }
        sc = g_static_ptr[dev];
        bad = g_static_bad_ptr[dev];
    }
    ddm_status st = upload_tables(ctx);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    Win<float> wf = make_win<float>(ctx, tau_lo, tau_hi);
    Win<double> wd = make_win<double>(ctx, tau_lo, tau_hi);
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_static_prep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_xy, d_x, n, sc, bad);
    k_static_dense<<<(unsigned)((n + ST_T - 1) / ST_T), ST_T, 0, s>>>(ctx->kf, ctx->kd, wf, wd, ctx->prm.quad_near, sc, d_x, n, d_y, bad);
    prof_end(ctx, 7, 2);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}
