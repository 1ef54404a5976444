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
struct GLTab {
    float xn[MAXGL], wn[MAXGL];   // near rule (fluid source), quad_near points
    float xf[3], wf[3];           // far rule, 3 points
    float xc[MAXGL], wc[MAXGL];   // P2M rule, n_cheb points
    float cheb[DDM_MAX_CHEB], bw[DDM_MAX_CHEB];
    int nn, nc;
};
__constant__ GLTab c_gl;

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

// Chebyshev cardinal functions S_n(xi_a, x) = l_a(x) at the roots of T_n,
// barycentric form (stable also slightly outside [-1, 1]).
template <int NMAX>
__device__ __forceinline__ void cardinal(float x, int n, float *out) {
    float s = 0.f;
    int hit = -1;
    for (int j = 0; j < n; ++j) {
        float d = x - c_gl.cheb[j];
        if (fabsf(d) < 1e-7f) hit = j;
        float v = c_gl.bw[j] / d;
        out[j] = v;
        s += v;
    }
    if (hit >= 0) {
        for (int j = 0; j < n; ++j) out[j] = (j == hit) ? 1.f : 0.f;
        return;
    }
    float is = 1.f / s;
    for (int j = 0; j < n; ++j) out[j] *= is;
}

// ----------------------------------------------------------------- charges
__global__ void k_charges(const double *x, const int64_t *perm, const float4 *frame, int64_t n, float4 *chg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t e = perm[i];
    float4 f = frame[i];
    float Ds = (float)x[e], Dn = (float)x[n + e], Dq = (float)x[2 * n + e];
    // D = Ds t + Dn n, n = (-ty, tx)
    chg[i] = make_float4(Ds * f.x - Dn * f.y, Ds * f.y + Dn * f.x, Dq, 0.f);
}

// --------------------------------------------------------- own element (FP64)
__global__ void k_self(KConst<double> k, Win<double> w, const double *x, const double *xy, int64_t n, double scale,
                       int overwrite, double *y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double dx = xy[2 * n + e] - xy[e], dy = xy[3 * n + e] - xy[n + e];
    double L = hypot(dx, dy);
    double o[3];
    self_field(k, w, 0.5 * L, dx / L, dy / L, x[e], x[n + e], x[2 * n + e], o);
    for (int r = 0; r < 3; ++r) {
        double v = scale * o[r];
        if (overwrite) y[r * n + e] = v; else y[r * n + e] += v;
    }
}

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

// own element through cached 3x3 blocks (caller order)
__global__ void k_self_apply(const double *blk, const double *x, int64_t n, double scale, int overwrite, double *y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double *B = blk + 9 * e;
    double a = x[e], b = x[n + e], c = x[2 * n + e];
    for (int r = 0; r < 3; ++r) {
        double v = scale * (B[3 * r] * a + B[3 * r + 1] * b + B[3 * r + 2] * c);
        if (overwrite) y[r * n + e] = v; else y[r * n + e] += v;
    }
}

// ---------------------------------------------------------------------- P2M
constexpr int P2M_T = 128;
__global__ void __launch_bounds__(P2M_T) k_p2m(const int32_t *cstart, const int32_t *cend, int64_t loff,
                                               const float4 *grel, const float4 *frame, const float4 *chg,
                                               float hL, int n, float *W) {
    __shared__ float sx[P2M_T][DDM_MAX_CHEB], sy[P2M_T][DDM_MAX_CHEB], wd[P2M_T][4];
    int64_t cell = loff + blockIdx.x;
    int s0 = cstart[cell], s1 = cend[cell];
    int nq = c_gl.nc, n2 = n * n;
    int npts = (s1 - s0) * nq;
    float acc[8];
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    float ih = 1.f / hL;
    for (int base = 0; base < npts; base += P2M_T) {
        int p = base + threadIdx.x;
        if (p < npts) {
            int e = s0 + p / nq, g = p % nq;
            float4 r = grel[e], f = frame[e], c = chg[e];
            float xi = c_gl.xc[g];
            float px = 0.5f * (r.x + r.z) + xi * f.z * f.x, py = 0.5f * (r.y + r.w) + xi * f.z * f.y;
            cardinal<DDM_MAX_CHEB>(px * ih, n, sx[threadIdx.x]);
            cardinal<DDM_MAX_CHEB>(py * ih, n, sy[threadIdx.x]);
            float wt = c_gl.wc[g] * f.z;           // ds = a dxi
            float nx = -f.y, ny = f.x;
            wd[threadIdx.x][0] = wt * c.x * nx;
            wd[threadIdx.x][1] = wt * c.y * ny;
            wd[threadIdx.x][2] = wt * 0.5f * (c.x * ny + c.y * nx);
            wd[threadIdx.x][3] = wt * c.z;
        }
        __syncthreads();
        int cnt = min(P2M_T, npts - base);
        for (int ent = threadIdx.x, slot = 0; ent < n2 && slot < 2; ent += P2M_T, ++slot) {
            int a = ent / n, b = ent % n;
            float s0_ = 0, s1_ = 0, s2_ = 0, s3_ = 0;
            for (int q = 0; q < cnt; ++q) {
                float v = sx[q][a] * sy[q][b];
                s0_ += v * wd[q][0]; s1_ += v * wd[q][1]; s2_ += v * wd[q][2]; s3_ += v * wd[q][3];
            }
            acc[4 * slot] += s0_; acc[4 * slot + 1] += s1_; acc[4 * slot + 2] += s2_; acc[4 * slot + 3] += s3_;
        }
        __syncthreads();
    }
    float *Wc = W + cell * 4 * n2;
    for (int ent = threadIdx.x, slot = 0; ent < n2 && slot < 2; ent += P2M_T, ++slot)
        for (int c = 0; c < 4; ++c) Wc[c * n2 + ent] = acc[4 * slot + c];
}

// ---------------------------------------------------------------------- M2M
// one block per child cell; adds S_n(ybar^parent, ybar^child) W^child to the parent
__global__ void k_m2m(int64_t off, const int32_t *cix, const int32_t *ciy, const int32_t *parent,
                      const float *T, int n, float *W) {
    extern __shared__ float sm[];
    float *wc = sm, *tmp = sm + 4 * n * n;
    int64_t cell = off + blockIdx.x;
    int n2 = n * n;
    const float *Wc = W + cell * 4 * n2;
    for (int i = threadIdx.x; i < 4 * n2; i += blockDim.x) wc[i] = Wc[i];
    __syncthreads();
    const float *Tx = T + ((cix[cell] & 1) ? n2 : 0), *Ty = T + ((ciy[cell] & 1) ? n2 : 0);
    // tmp[c][a][b'] = sum_a' Tx[a][a'] wc[c][a'][b']
    for (int i = threadIdx.x; i < 4 * n2; i += blockDim.x) {
        int c = i / n2, a = (i / n) % n, b = i % n;
        float s = 0;
        for (int ap = 0; ap < n; ++ap) s += Tx[a * n + ap] * wc[c * n2 + ap * n + b];
        tmp[i] = s;
    }
    __syncthreads();
    float *Wp = W + (int64_t)parent[cell] * 4 * n2;
    for (int i = threadIdx.x; i < 4 * n2; i += blockDim.x) {
        int c = i / n2, a = (i / n) % n, b = i % n;
        float s = 0;
        for (int bp = 0; bp < n; ++bp) s += Ty[b * n + bp] * tmp[c * n2 + a * n + bp];
        atomicAdd(&Wp[i], s);
    }
}

// ---------------------------------------------------------------------- L2L
// one block per child cell: f^child += S_n(xbar^child in parent) f^parent
__global__ void k_l2l(int64_t off, const int32_t *cix, const int32_t *ciy, const int32_t *parent,
                      const float *T, int n, float *F) {
    extern __shared__ float sm[];
    float *fp = sm, *tmp = sm + 4 * n * n;
    int64_t cell = off + blockIdx.x;
    int n2 = n * n;
    const float *Fp = F + (int64_t)parent[cell] * 4 * n2;
    for (int i = threadIdx.x; i < 4 * n2; i += blockDim.x) fp[i] = Fp[i];
    __syncthreads();
    const float *Tx = T + ((cix[cell] & 1) ? n2 : 0), *Ty = T + ((ciy[cell] & 1) ? n2 : 0);
    // child node a' takes sum_a T[a][a'] (transpose of M2M)
    for (int i = threadIdx.x; i < 4 * n2; i += blockDim.x) {
        int c = i / n2, ap = (i / n) % n, b = i % n;
        float s = 0;
        for (int a = 0; a < n; ++a) s += Tx[a * n + ap] * fp[c * n2 + a * n + b];
        tmp[i] = s;
    }
    __syncthreads();
    float *Fc = F + cell * 4 * n2;
    for (int i = threadIdx.x; i < 4 * n2; i += blockDim.x) {
        int c = i / n2, ap = (i / n) % n, bp = i % n;
        float s = 0;
        for (int b = 0; b < n; ++b) s += Ty[b * n + bp] * tmp[c * n2 + ap * n + b];
        Fc[i] += s;
    }
}

// ---------------------------------------------------------------------- M2L
// One block (4 warps) per target cell at levels >= 2; the warps take
// interleaved entries of the interaction list, each lane owns NPL target
// nodes and evaluates the kernel against all n^2 source nodes of the entry
// (weights staged in shared memory); the four warps' sums are reduced in
// shared memory at the end.
struct LevelTab {
    int64_t off[DDM_MAX_LEVELS + 2];
    int L;
};
constexpr int M2L_W = 4;
template <int NPL>
__global__ void __launch_bounds__(32 * M2L_W) k_m2l(KConst<float> k, Win<float> w, LevelTab lt, int64_t first,
                                                   const int32_t *iloff, const int32_t *ilidx, const int32_t *cix,
                                                   const int32_t *ciy, double h0, int n, const float *W, float *F) {
    extern __shared__ float sm[];            // M2L_W x 4 n^2 (weights, then partial sums)
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int n2 = n * n;
    float *sw = sm + wid * 4 * n2;
    int64_t cell = first + blockIdx.x;
    int lvl = 0;
    while (lvl < lt.L && cell >= lt.off[lvl + 1]) ++lvl;
    float h = (float)(h0 / (double)(1 << lvl)), wl = 2.f * h;
    int ixI = cix[cell], iyI = ciy[cell];
    float acc[NPL][4];
    float tx[NPL], ty[NPL];
#pragma unroll
    for (int r = 0; r < NPL; ++r) {
        int m = lane + 32 * r;
        acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
        tx[r] = m < n2 ? h * c_gl.cheb[m / n] : 0.f;
        ty[r] = m < n2 ? h * c_gl.cheb[m % n] : 0.f;
    }
    for (int q = iloff[cell] + wid; q < iloff[cell + 1]; q += M2L_W) {
        int32_t J = ilidx[q];
        const float *WJ = W + (int64_t)J * 4 * n2;
        __syncwarp();
        for (int i = lane; i < 4 * n2; i += 32) sw[i] = WJ[i];
        __syncwarp();
        float ox = wl * (float)(ixI - cix[J]), oy = wl * (float)(iyI - ciy[J]);
        for (int ap = 0; ap < n; ++ap) {
            float sx = ox - h * c_gl.cheb[ap];
            for (int bp = 0; bp < n; ++bp) {
                int mp = ap * n + bp;
                float sy = oy - h * c_gl.cheb[bp];
                float w0 = sw[mp], w1 = sw[n2 + mp], w2 = sw[2 * n2 + mp], w3 = sw[3 * n2 + mp];
#pragma unroll
                for (int r = 0; r < NPL; ++r)
                    if (lane + 32 * r < n2) pot_kernel<float>(k, tx[r] + sx, ty[r] + sy, w0, w1, w2, w3, w, acc[r]);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NPL; ++r) {
        int m = lane + 32 * r;
        if (m < n2)
            for (int c = 0; c < 4; ++c) sm[wid * 4 * n2 + c * n2 + m] = acc[r][c];
    }
    __syncthreads();
    float *Fc = F + cell * 4 * n2;
    for (int i = threadIdx.x; i < 4 * n2; i += 32 * M2L_W) {
        float v = 0.f;
        for (int ww = 0; ww < M2L_W; ++ww) v += sm[ww * 4 * n2 + i];
        Fc[i] = v;
    }
}

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
    float zx = 2.f * h * dx + h * (c_gl.cheb[m / n] - c_gl.cheb[mp / n]);
    float zy = 2.f * h * dy + h * (c_gl.cheb[m % n] - c_gl.cheb[mp % n]);
    float *K = ops + (int64_t)key * 16 * n2 * n2;
    int ld = 4 * n2;
    for (int ci = 0; ci < 4; ++ci) {
        float a[4] = {0, 0, 0, 0};
        pot_kernel<float>(k, zx, zy, ci == 0, ci == 1, ci == 2, ci == 3, w, a);
        for (int co = 0; co < 4; ++co) K[(int64_t)(co * n2 + m) * ld + ci * n2 + mp] = a[co];
    }
}

// One work item = one (level, offset) group's column tile of up to 64
// interaction pairs; blockIdx.y picks a 128-row slice of the 4n^2 operator
// rows.  256 threads, 8 x 4 register tile each, BK = 16, double-buffered
// shared memory; results are added to the targets' local expansions.
constexpr int GM_BM = 128, GM_BN = 64, GM_BK = 16;
__global__ void __launch_bounds__(256) k_m2l_gemm(const int2 *work, const int32_t *koff, const int2 *pairs, int n,
                                                  const float *ops, const float *W, float *F) {
    __shared__ __align__(16) float sK[2][GM_BK][GM_BM];
    __shared__ __align__(16) float sB[2][GM_BK][GM_BN];
    __shared__ int sI[GM_BN], sJ[GM_BN];
    int2 wk = work[blockIdx.x];
    int key = wk.x, p0 = wk.y, p1 = min(koff[key + 1], p0 + GM_BN);
    int n2 = n * n, ld = 4 * n2;
    int r0 = blockIdx.y * GM_BM;
    const float *K = ops + (int64_t)key * 16 * n2 * n2;
    int tid = threadIdx.x;
    if (tid < GM_BN) {
        int p = p0 + tid;
        sI[tid] = p < p1 ? pairs[p].x : -1;
        sJ[tid] = p < p1 ? pairs[p].y : -1;
    }
    __syncthreads();
    // loaders: K tile 128 x 16 -> each thread 8 consecutive k of one row;
    // B tile 16 x 64 -> each thread 4 consecutive k of one column
    int kr = tid >> 1, kk0 = (tid & 1) * 8;
    int bj = tid >> 2, bk0 = (tid & 3) * 4;
    int Jb = sJ[bj];
    int tr = (tid >> 4) * 8, tc = (tid & 15) * 4;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    int nsteps = ld / GM_BK;
    for (int st = 0; st <= nsteps; ++st) {
        int buf = st & 1;
        if (st < nsteps) {       // stage step st into buffer buf
            int k0 = st * GM_BK, row = r0 + kr;
            if (row < ld) {
                const float *src = K + (int64_t)row * ld + k0 + kk0;
                float4 v0 = *(const float4 *)src, v1 = *(const float4 *)(src + 4);
                sK[buf][kk0 + 0][kr] = v0.x; sK[buf][kk0 + 1][kr] = v0.y;
                sK[buf][kk0 + 2][kr] = v0.z; sK[buf][kk0 + 3][kr] = v0.w;
                sK[buf][kk0 + 4][kr] = v1.x; sK[buf][kk0 + 5][kr] = v1.y;
                sK[buf][kk0 + 6][kr] = v1.z; sK[buf][kk0 + 7][kr] = v1.w;
            } else {
                for (int q = 0; q < 8; ++q) sK[buf][kk0 + q][kr] = 0.f;
            }
            if (Jb >= 0) {
                float4 v = *(const float4 *)(W + (int64_t)Jb * ld + k0 + bk0);
                sB[buf][bk0 + 0][bj] = v.x; sB[buf][bk0 + 1][bj] = v.y;
                sB[buf][bk0 + 2][bj] = v.z; sB[buf][bk0 + 3][bj] = v.w;
            } else {
                for (int q = 0; q < 4; ++q) sB[buf][bk0 + q][bj] = 0.f;
            }
        }
        if (st > 0) {            // compute step st - 1 from the other buffer
            int cur = buf ^ 1;
#pragma unroll
            for (int kk = 0; kk < GM_BK; ++kk) {
                float4 a0 = *(const float4 *)&sK[cur][kk][tr], a1 = *(const float4 *)&sK[cur][kk][tr + 4];
                float4 b0 = *(const float4 *)&sB[cur][kk][tc];
                float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                float bb[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int I = sI[tc + j];
        if (I < 0) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int row = r0 + tr + i;
            if (row < ld) atomicAdd(&F[(int64_t)I * ld + row], acc[i][j]);
        }
    }
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
    for (int side = 0; side < 2; ++side) {
        float ct = side == 0 ? w.ct_hi : w.ct_lo;
        if (ct <= 0.f) continue;
        float s = side == 0 ? 1.f : -1.f;
        float x2 = zx * zx, y2 = zy * zy, r2 = x2 + y2;
        float ir2 = 1.f / r2;
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

// near/far element integral of one source element at target m (target
// frame coordinates); self pairs are excluded by the caller.  PRECISE: the
// DD part of every pair in FP64 (closed form near, Gauss rule far) - the
// element contributions along a fracture nearly cancel for smooth openings,
// by a factor that grows with the elements per fracture, so residuals need
// FP64 here; the fluid-source part stays FP32.
template <bool PRECISE>
__device__ __forceinline__ void pair_field(const KConst<float> &k, const KConst<double> &kd, const Win<float> &w,
                                           const Win<double> &wd, float mx, float my, const SrcTile &s,
                                           float acc[4], double accd[4]) {
    float cxs = 0.5f * (s.x0 + s.x1), cys = 0.5f * (s.y0 + s.y1);
    float dx = mx - cxs, dy = my - cys;
    float r2 = dx * dx + dy * dy;
    bool far = r2 > 64.f * s.a * s.a;
    if (PRECISE) {
        if (far) {
            double nx = -(double)s.ty, ny = (double)s.tx;
            double Pxx = s.Dx * nx, Pyy = s.Dy * ny, Pxy = 0.5 * (s.Dx * ny + s.Dy * nx);
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                double sg = (double)c_gl.xf[g] * s.a, wt = (double)c_gl.wf[g] * s.a;
                pot_kernel<double>(kd, dx - sg * s.tx, dy - sg * s.ty, wt * Pxx, wt * Pyy, wt * Pxy, 0.0, wd, accd);
            }
        } else {
            disl_field<double>(kd, (double)(mx - s.x0), (double)(my - s.y0), (double)s.Dx, (double)s.Dy, wd, 1.0, accd);
            disl_field<double>(kd, (double)(mx - s.x1), (double)(my - s.y1), (double)s.Dx, (double)s.Dy, wd, -1.0, accd);
        }
        if (s.q != 0.f) {
            if (far) {
#pragma unroll
                for (int g = 0; g < 3; ++g) {
                    float sg = c_gl.xf[g] * s.a, wt = c_gl.wf[g] * s.a;
                    q_point(k, dx - sg * s.tx, dy - sg * s.ty, wt * s.q, w, acc);
                }
            } else {
                for (int g = 0; g < c_gl.nn; ++g) {
                    float sg = c_gl.xn[g] * s.a, wt = c_gl.wn[g] * s.a;
                    q_point(k, dx - sg * s.tx, dy - sg * s.ty, wt * s.q, w, acc);
                }
            }
        }
        return;
    }
    if (far) {
        // far: 3-point Gauss rule of the point kernel
        float nx = -s.ty, ny = s.tx;
        float Pxx = s.Dx * nx, Pyy = s.Dy * ny, Pxy = 0.5f * (s.Dx * ny + s.Dy * nx);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            float sg = c_gl.xf[g] * s.a, wt = c_gl.wf[g] * s.a;
            pot_kernel<float>(k, dx - sg * s.tx, dy - sg * s.ty, wt * Pxx, wt * Pyy, wt * Pxy, wt * s.q, w, acc);
        }
    } else {
        disl_field<float>(k, mx - s.x0, my - s.y0, s.Dx, s.Dy, w, 1.f, acc);
        disl_field<float>(k, mx - s.x1, my - s.y1, s.Dx, s.Dy, w, -1.f, acc);
        if (s.q != 0.f) {
            for (int g = 0; g < c_gl.nn; ++g) {
                float sg = c_gl.xn[g] * s.a, wt = c_gl.wn[g] * s.a;
                q_point(k, dx - sg * s.tx, dy - sg * s.ty, wt * s.q, w, acc);
            }
        }
    }
}

// Near field + L2P.  One warp per target: the lanes take the sources of the
// target leaf's neighbour leaves (self + up to 8; about 50 sources at the
// usual depths) in a strided loop, so nearly every lane has a pair and there
// are as many warps as targets.  Each lane sums its pairs in FP32, the warp
// then reduces in FP64; L2P is split over the lanes by Chebyshev node and
// reduced the same way.
constexpr int NEAR_W = 8;
constexpr int NEAR_T = 32 * NEAR_W;
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
template <bool PRECISE>
__global__ void __launch_bounds__(NEAR_T) k_near(KConst<float> k, KConst<double> kd, Win<float> w, Win<double> wd,
                                                 int64_t loff, const int32_t *cstart, const int32_t *cend,
                                                 const int32_t *cix, const int32_t *ciy, const int32_t *nboff,
                                                 const int32_t *nbidx, const int32_t *elem_leaf, const float4 *grel,
                                                 const float4 *frame, const float4 *chg, const int64_t *perm,
                                                 float wL, int n, const float *F, int use_far, int64_t N,
                                                 double scale, double *y) {
    __shared__ int sst[NEAR_W][9], spre[NEAR_W][10];
    __shared__ float sox[NEAR_W][9], soy[NEAR_W][9];
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t ti = (int64_t)blockIdx.x * NEAR_W + wid;
    if (ti >= N) return;                      // whole warp leaves together
    int32_t leaf = elem_leaf[ti];
    int64_t cell = loff + leaf;
    int ix = cix[cell], iy = ciy[cell];
    int q0 = nboff[leaf], nq = nboff[leaf + 1] - q0;
    if (lane == 0) {
        int run = 0;
        for (int q = 0; q < nq; ++q) {
            int64_t J = loff + nbidx[q0 + q];
            sst[wid][q] = cstart[J];
            spre[wid][q] = run;
            run += cend[J] - cstart[J];
            sox[wid][q] = wL * (float)(cix[J] - ix);
            soy[wid][q] = wL * (float)(ciy[J] - iy);
        }
        spre[wid][nq] = run;
    }
    __syncwarp();
    float4 rt = grel[ti];
    float mx = 0.5f * (rt.x + rt.z), my = 0.5f * (rt.y + rt.w);
    int S = spre[wid][nq];
    float acc[4] = {0, 0, 0, 0};
    double accd[4] = {0, 0, 0, 0};
    int q = 0;
    for (int c = lane; c < S; c += 32) {
        while (c >= spre[wid][q + 1]) ++q;
        int sj = sst[wid][q] + (c - spre[wid][q]);
        if (sj == (int)ti) continue;
        float4 r = grel[sj], f = frame[sj], cg = chg[sj];
        float ox = sox[wid][q], oy = soy[wid][q];
        SrcTile st;
        st.x0 = r.x + ox; st.y0 = r.y + oy; st.x1 = r.z + ox; st.y1 = r.w + oy;
        st.Dx = cg.x; st.Dy = cg.y; st.q = cg.z; st.a = f.z; st.tx = f.x; st.ty = f.y; st.idx = sj;
        pair_field<PRECISE>(k, kd, w, wd, mx, my, st, acc, accd);
    }
    for (int c = 0; c < 4; ++c) accd[c] += (double)acc[c];
    if (use_far) {
        // L2P: lane handles nodes m = lane, lane + 32, ...
        float hL = 0.5f * wL;
        float xh = mx / hL, yh = my / hL;
        int n2 = n * n;
        float sx = 0.f, sy = 0.f;
        int hx = -1, hy = -1;
        for (int j = 0; j < n; ++j) {             // barycentric denominators
            float dxj = xh - c_gl.cheb[j], dyj = yh - c_gl.cheb[j];
            if (fabsf(dxj) < 1e-7f) hx = j;
            if (fabsf(dyj) < 1e-7f) hy = j;
            sx += c_gl.bw[j] / dxj;
            sy += c_gl.bw[j] / dyj;
        }
        const float *Fc = F + cell * 4 * n2;
        float f4[4] = {0, 0, 0, 0};
        for (int m = lane; m < n2; m += 32) {
            int a = m / n, bb = m % n;
            float la = hx >= 0 ? (a == hx ? 1.f : 0.f) : c_gl.bw[a] / (xh - c_gl.cheb[a]) / sx;
            float lb = hy >= 0 ? (bb == hy ? 1.f : 0.f) : c_gl.bw[bb] / (yh - c_gl.cheb[bb]) / sy;
            float v = la * lb;
            f4[0] += v * Fc[m]; f4[1] += v * Fc[n2 + m]; f4[2] += v * Fc[2 * n2 + m]; f4[3] += v * Fc[3 * n2 + m];
        }
        for (int c = 0; c < 4; ++c) accd[c] += (double)f4[c];
    }
    for (int c = 0; c < 4; ++c) accd[c] = warp_sum(accd[c]);
    if (lane != 0) return;
    float4 f = frame[ti];
    double ss, sn;
    to_local<double>((double)f.x, (double)f.y, accd, ss, sn);
    int64_t e = perm[ti];
    y[e] += scale * ss;
    y[N + e] += scale * sn;
    y[2 * N + e] += scale * accd[3];
}

// -------------------------------------------------------------------- dense
constexpr int DN_T = 128;
template <bool PRECISE>
__global__ void __launch_bounds__(DN_T) k_dense(KConst<float> k, KConst<double> kd, Win<float> w, Win<double> wd, int64_t loff, const int32_t *elem_leaf,
                                                const int32_t *cix, const int32_t *ciy, const float4 *grel,
                                                const float4 *frame, const float4 *chg, const int64_t *perm,
                                                float wL, int64_t N, int64_t chunk, double scale, double *y) {
    __shared__ SrcTile tile[DN_T];
    __shared__ int sjx[DN_T], sjy[DN_T];
    int64_t ti = blockIdx.x * (int64_t)DN_T + threadIdx.x;
    bool act = ti < N;
    float mx = 0, my = 0, ttx = 1, tty = 0;
    int ixI = 0, iyI = 0;
    if (act) {
        float4 r = grel[ti], f = frame[ti];
        mx = 0.5f * (r.x + r.z); my = 0.5f * (r.y + r.w);
        ttx = f.x; tty = f.y;
        int32_t c = elem_leaf[ti];
        ixI = cix[loff + c]; iyI = ciy[loff + c];
    }
    double accd[4] = {0, 0, 0, 0};
    int64_t s0 = blockIdx.y * chunk;
    int64_t s1 = s0 + chunk < N ? s0 + chunk : N;
    for (int64_t sb = s0; sb < s1; sb += DN_T) {
        __syncthreads();
        int64_t sj = sb + threadIdx.x;
        if (sj < s1) {
            float4 r = grel[sj], f = frame[sj], c = chg[sj];
            SrcTile s;
            s.x0 = r.x; s.y0 = r.y; s.x1 = r.z; s.y1 = r.w;
            s.Dx = c.x; s.Dy = c.y; s.q = c.z; s.a = f.z; s.tx = f.x; s.ty = f.y; s.idx = (int)sj;
            tile[threadIdx.x] = s;
            int32_t cl = elem_leaf[sj];
            sjx[threadIdx.x] = cix[loff + cl];
            sjy[threadIdx.x] = ciy[loff + cl];
        }
        __syncthreads();
        int cnt = (int)(s1 - sb < DN_T ? s1 - sb : DN_T);
        if (act) {
            float acc[4] = {0, 0, 0, 0};          // one tile in FP32, tiles summed in FP64
            for (int j = 0; j < cnt; ++j) {
                if (tile[j].idx == (int)ti) continue;
                SrcTile s = tile[j];
                float ox = wL * (float)(sjx[j] - ixI), oy = wL * (float)(sjy[j] - iyI);
                s.x0 += ox; s.y0 += oy; s.x1 += ox; s.y1 += oy;
                pair_field<PRECISE>(k, kd, w, wd, mx, my, s, acc, accd);
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

}  // namespace

// ------------------------------------------------------------------- host
// The Gauss / Chebyshev tables live in __constant__ memory, which is global
// to the device: the last uploaded (n_cheb, quad_near) is tracked process
// wide, and contexts that use different values on one device must not run
// concurrently.
static std::mutex g_tab_mu;
static int g_last_n[64], g_last_q[64];
static bool g_tab_init = false;
ddm_status upload_tables(ddm_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (!g_tab_init) {
        for (int i = 0; i < 64; ++i) g_last_n[i] = g_last_q[i] = -1;
        g_tab_init = true;
    }
    int n = ctx->prm.n_cheb, nq = ctx->prm.quad_near, dv = ctx->device & 63;
    if (n == g_last_n[dv] && nq == g_last_q[dv]) return DDM_OK;
    GLTab h;
    memset(&h, 0, sizeof(h));
    double x[MAXGL], wt[MAXGL];
    gauss_legendre(nq, x, wt);
    for (int i = 0; i < nq; ++i) { h.xn[i] = (float)x[i]; h.wn[i] = (float)wt[i]; }
    h.nn = nq;
    gauss_legendre(3, x, wt);
    for (int i = 0; i < 3; ++i) { h.xf[i] = (float)x[i]; h.wf[i] = (float)wt[i]; }
    gauss_legendre(n, x, wt);
    for (int i = 0; i < n; ++i) { h.xc[i] = (float)x[i]; h.wc[i] = (float)wt[i]; }
    h.nc = n;
    for (int j = 0; j < n; ++j) {
        double th = (2 * j + 1) * M_PI / (2.0 * n);
        h.cheb[j] = (float)cos(th);
        h.bw[j] = (float)(((j & 1) ? -1.0 : 1.0) * sin(th));
    }
    DDM_CUDA_TRY(ctx, cudaMemcpyToSymbolAsync(c_gl, &h, sizeof(h), 0, cudaMemcpyHostToDevice, ctx->stream));
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    g_last_n[dv] = n; g_last_q[dv] = nq;
    return DDM_OK;
}

ddm_status ensure_workspace(ddm_ctx *ctx, ddm_tree *t) {
    int n = ctx->prm.n_cheb;
    if (t->ncheb_alloc == n && t->W) return DDM_OK;
    dfree(t->W, t->stream);
    dfree(t->Fl, t->stream);
    t->W = t->Fl = nullptr;
    size_t sz = (size_t)t->n_cells * 4 * n * n * sizeof(float);
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
    return w;
}

ddm_status self_blocks(ddm_ctx *ctx, ddm_tree *t, double dt) {
    if (t->self_dt == dt) return DDM_OK;
    int64_t n = t->n;
    k_self_blocks<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->kd, make_win<double>(ctx, 0.0, dt), t->xy_caller, n,
                                                            t->self_blk);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    t->self_dt = dt;
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
    int n = ctx->prm.n_cheb, n2 = n * n;
    const int TB = 256;
    KConst<float> kf = ctx->kf;
    Win<float> wf = make_win<float>(ctx, lo, hi);
    Win<double> wd = make_win<double>(ctx, lo, hi);
    prof_begin(ctx, 0);
    k_charges<<<(N + TB - 1) / TB, TB, 0, s>>>(x, t->perm, t->g_frame, N, t->chg);
    prof_end(ctx, 0, 1);
    // own elements (FP64 closed form), caller order
    prof_begin(ctx, 1);
    {
        // own-element blocks of this time window, computed once and cached
        int slot = -1;
        for (int k = 0; k < 4; ++k)
            if (t->win_blk[k] && t->win_lo[k] == lo && t->win_hi[k] == hi) slot = k;
        if (slot < 0) {
            slot = t->win_next;
            t->win_next = (t->win_next + 1) % 4;
            if (!t->win_blk[slot]) DDM_CUDA_TRY(ctx, dalloc(&t->win_blk[slot], 9 * N * sizeof(double), t->stream));
            k_self_blocks<<<(N + TB - 1) / TB, TB, 0, s>>>(ctx->kd, wd, t->xy_caller, N, t->win_blk[slot]);
            t->win_lo[slot] = lo;
            t->win_hi[slot] = hi;
        }
        k_self_apply<<<(N + TB - 1) / TB, TB, 0, s>>>(t->win_blk[slot], x, N, scale, accumulate ? 0 : 1, y);
    }
    prof_end(ctx, 1, 1);
    int L = t->depth;
    int64_t loff = t->lvl_off[L], nleaf = t->lvl_off[L + 1] - loff;
    float wL = (float)(2.0 * t->h0 / (double)(1 << L));
    if (mode == DDM_MODE_DENSE) {
        int64_t tiles = (N + DN_T - 1) / DN_T;
        int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + tiles - 1) / tiles, (N + DN_T - 1) / DN_T));
        int64_t chunk = ((N + chunks - 1) / chunks + DN_T - 1) / DN_T * DN_T;
        chunks = (N + chunk - 1) / chunk;
        prof_begin(ctx, 7);
        auto kdn = precise ? k_dense<true> : k_dense<false>;
        kdn<<<dim3((unsigned)tiles, (unsigned)chunks), DN_T, 0, s>>>(kf, ctx->kd, wf, wd, loff, t->elem_leaf, t->cell_ix, t->cell_iy,
                                                                        t->g_rel, t->g_frame, t->chg, t->perm, wL, N,
                                                                        chunk, scale, y);
        prof_end(ctx, 7, 1);
        DDM_CUDA_TRY(ctx, cudaGetLastError());
        return DDM_OK;
    }
    int use_far = L >= 2;
    if (use_far) {
        float hL = 0.5f * wL;
        // upward pass
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(t->W, 0, (size_t)t->n_cells * 4 * n2 * sizeof(float), s));
        prof_begin(ctx, 2);
        k_p2m<<<(unsigned)nleaf, P2M_T, 0, s>>>(t->cell_start, t->cell_end, loff, t->g_rel, t->g_frame, t->chg, hL, n,
                                                t->W);
        prof_end(ctx, 2, 1);
        size_t sm2 = 8 * n2 * sizeof(float);
        prof_begin(ctx, 3);
        for (int l = L; l >= 3; --l) {
            int64_t off = t->lvl_off[l], nc = t->lvl_off[l + 1] - off;
            k_m2m<<<(unsigned)nc, 128, sm2, s>>>(off, t->cell_ix, t->cell_iy, t->cell_parent, ctx->cheb_T, n, t->W);
        }
        prof_end(ctx, 3, L - 2);
        // M2L on every level >= 2 in one launch
        LevelTab lt;
        for (int l = 0; l <= L + 1 && l < DDM_MAX_LEVELS + 2; ++l) lt.off[l] = t->lvl_off[l];
        lt.L = L;
        int64_t first = t->lvl_off[2], ncm = t->lvl_off[L + 1] - first;
        prof_begin(ctx, 4);
        {
            int nk = t->n_keys;
            size_t opsz = (size_t)nk * 16 * n2 * n2;
            if (t->ops_n != n || !t->m2l_ops) {
                dfree(t->m2l_ops, t->stream);
                t->m2l_ops = nullptr;
                DDM_CUDA_TRY(ctx, dalloc(&t->m2l_ops, opsz * sizeof(float), t->stream));
                t->ops_n = n;
                t->ops_lo = t->ops_hi = -1.0;
            }
            if (t->ops_lo != lo || t->ops_hi != hi) {
                dim3 g((unsigned)((n2 * n2 + 127) / 128), (unsigned)nk);
                k_m2l_ops<<<g, 128, 0, s>>>(kf, wf, L, t->h0, n, t->mk_off, t->m2l_ops);
                t->ops_lo = lo;
                t->ops_hi = hi;
                prof_end(ctx, 4, 1);
                prof_begin(ctx, 4);
            }
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(t->Fl, 0, (size_t)t->n_cells * 4 * n2 * sizeof(float), s));
            if (t->n_work > 0) {
                dim3 g((unsigned)t->n_work, (unsigned)((4 * n2 + GM_BM - 1) / GM_BM));
                k_m2l_gemm<<<g, 256, 0, s>>>(t->mk_work, t->mk_off, t->mk_pair, n, t->m2l_ops, t->W, t->Fl);
            }
        }
        prof_end(ctx, 4, 1);
        // downward pass
        prof_begin(ctx, 5);
        for (int l = 3; l <= L; ++l) {
            int64_t off = t->lvl_off[l], nc = t->lvl_off[l + 1] - off;
            k_l2l<<<(unsigned)nc, 128, sm2, s>>>(off, t->cell_ix, t->cell_iy, t->cell_parent, ctx->cheb_T, n, t->Fl);
        }
        prof_end(ctx, 5, L - 2);
    }
    prof_begin(ctx, 6);
    auto knr = precise ? k_near<true> : k_near<false>;
    knr<<<(unsigned)((N + NEAR_W - 1) / NEAR_W), NEAR_T, 0, s>>>(
        kf, ctx->kd, wf, wd, loff, t->cell_start, t->cell_end, t->cell_ix, t->cell_iy, t->nb_off, t->nb_idx,
        t->elem_leaf, t->g_rel, t->g_frame, t->chg, t->perm, wL, n, t->Fl, use_far, N, scale, y);
    prof_end(ctx, 6, 1);
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
// and nothing in the array needs to start at zero.
// ---------------------------------------------------------------------------
namespace {
struct StaticElem {
    double2 mid;     // midpoint (FP64)
    float4 frame;    // tangent (x, y), half-length, unused
    float4 chg;      // global DD vector (x, y), fluid source, unused
};
static __device__ __align__(256) StaticElem g_static_scratch[DDM_STATIC_MAX_ELEMENTS];

std::mutex g_static_mu;
StaticElem *g_static_ptr[256] = {nullptr};   // device address of the array, per device

__global__ void k_static_prep(const double *xy, const double *x, int64_t n, StaticElem *sc) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double ax = xy[e], ay = xy[n + e], bx = xy[2 * n + e], by = xy[3 * n + e];
    double L = hypot(bx - ax, by - ay), tx = (bx - ax) / L, ty = (by - ay) / L;
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
                                                       Win<double> wd, const StaticElem *sc, const double *x,
                                                       int64_t n, double *y) {
    __shared__ StaticElem tile[ST_T];
    int64_t ti = blockIdx.x * (int64_t)ST_T + threadIdx.x;
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
                pair_field<false>(k, kd, w, wd, 0.f, 0.f, st, acc, accd);
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
    if (!ctx || !d_xy || !d_x || !d_y || d_x == d_y)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: bad arguments");
    if (n <= 0 || n > DDM_STATIC_MAX_ELEMENTS)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: n must be in [1, " +
                                             std::to_string(DDM_STATIC_MAX_ELEMENTS) + "], got " + std::to_string(n));
    if (!(tau_hi > tau_lo) || tau_lo < 0.0)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: need 0 <= tau_lo < tau_hi");
    int dev = 0;
    DDM_CUDA_TRY(ctx, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec_dense_static: device index out of range");
    StaticElem *sc = nullptr;
    {
        // set-up, once per device, with that device current: the host-side
        // name of the array is not a device address; ask the runtime for it
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess)
                return ctx_fail(ctx, DDM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_static_ptr[dev] = (StaticElem *)p;
        }
        sc = g_static_ptr[dev];
    }
    ddm_status st = upload_tables(ctx);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    Win<float> wf = make_win<float>(ctx, tau_lo, tau_hi);
    Win<double> wd = make_win<double>(ctx, tau_lo, tau_hi);
    k_static_prep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_xy, d_x, n, sc);
    k_static_dense<<<(unsigned)((n + ST_T - 1) / ST_T), ST_T, 0, s>>>(ctx->kf, ctx->kd, wf, wd, sc, d_x, n, d_y);
    prof_end(ctx, 7, 2);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}
