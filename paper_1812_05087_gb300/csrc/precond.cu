// Block-Jacobi preconditioner over fracture chains.
//
// Elements that share end points form chains (one fracture); the chains are
// cut into blocks of at most 64 elements at tree build.  For a time step dt
// each block's own influence matrix (all its element pairs: FP32 closed
// forms for the DD part on FP64 offsets, Gauss rule for the fluid source,
// the own element from the cached FP64 closed form) is assembled for the
// rows and unknowns of the system being solved and inverted on the device
// in FP32 (Gauss-Jordan with partial pivoting, one CTA per matrix held in
// registers); a preconditioner needs no more precision, and FP32 runs
// at 64x the FP64 rate.  Applying the preconditioner is
// one small dense product per block.  Elements that belong to no chain form
// 1-element blocks, i.e. the own-element 3x3 block Jacobi.
//
// Long chains (at least PC_MIN_BLOCKS blocks) add a coarse level: on each of
// their blocks, Legendre modes of degree < pc_modes in the block's element
// index, one set per unknown component, span the coarse space Z; the
// Galerkin matrix A_c = Z^T A Z (all element pairs of every pair of coarse
// blocks) is assembled and inverted on the device once per (dt, system),
// and the preconditioner becomes additive two-level,
// M^-1 = blockdiag^-1 + Z A_c^-1 Z^T.  Block Jacobi alone leaves the long-
// wavelength modes of a long fracture (and the coupling between parallel
// fractures) to the Krylov iteration, whose count then grows with the chain
// length; the coarse level carries them.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "kernel_math.cuh"

namespace {

// Gauss-Legendre, 8 points on [-1, 1] (fluid source between elements)
__constant__ double c_gl8x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                                 0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
__constant__ double c_gl8w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                                 0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

// per element (caller order): FP64 midpoint, FP32 tangent and half-length
struct PbGeo {
    double2 mid;
    float4 t;        // tx, ty, a, 0
};
__global__ void k_pb_geom(const double *xy, int64_t N, PbGeo *g) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    double ax = xy[e], ay = xy[N + e], bx = xy[2 * N + e], by = xy[3 * N + e];
    double L = hypot(bx - ax, by - ay);
    g[e].mid = make_double2(0.5 * (ax + bx), 0.5 * (ay + by));
    g[e].t = make_float4((float)((bx - ax) / L), (float)((by - ay) / L), (float)(0.5 * L), 0.f);
}

// rows (sigma_s, sigma_n, p) at element i's midpoint from unit (Ds, Dn, Dq)
// on element j != i: FP32 pair arithmetic on the FP64 midpoint offset (the
// preconditioner needs no more)
__device__ void pair_block(const KConst<float> &kf, const Win<float> &wf, const PbGeo &gi, const PbGeo &gj,
                           float out[3][3]) {
    float ox = (float)(gi.mid.x - gj.mid.x), oy = (float)(gi.mid.y - gj.mid.y);
    float tjx = gj.t.x, tjy = gj.t.y, a = gj.t.z, njx = -tjy, njy = tjx;
    float z1x = ox + a * tjx, z1y = oy + a * tjy, z2x = ox - a * tjx, z2y = oy - a * tjy;
    for (int c = 0; c < 2; ++c) {
        float Dx = c == 0 ? tjx : njx, Dy = c == 0 ? tjy : njy;
        float g[4] = {0, 0, 0, 0};
        disl_field<float>(kf, z1x, z1y, Dx, Dy, wf, 1.f, g);
        disl_field<float>(kf, z2x, z2y, Dx, Dy, wf, -1.f, g);
        float ss, sn;
        to_local<float>(gi.t.x, gi.t.y, g, ss, sn);
        out[0][c] = ss; out[1][c] = sn; out[2][c] = g[3];
    }
    // fluid source: 8-point Gauss rule of the point kernel along element j
    float g[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        float s = (float)c_gl8x[q] * a, wt = (float)c_gl8w[q] * a;
        float zx = ox - s * tjx, zy = oy - s * tjy;
        float ir2 = 1.f / (zx * zx + zy * zy);
        pot_transient<float>(kf, zx, zy, ir2, 0.f, 0.f, 0.f, wt, wf.g_hi, 4.f * wf.ct_hi, 1.f, g);
    }
    float ss, sn;
    to_local<float>(gi.t.x, gi.t.y, g, ss, sn);
    out[0][2] = ss; out[1][2] = sn; out[2][2] = g[3];
}

// assemble the system block of every preconditioner block:
// row (rc * m + i), column (cc * m + j), rc, cc < nc; RATE: row 1 = sigma_n + p;
// the own element from the cached FP64 3x3 blocks of the step
__global__ void k_pb_assemble(KConst<float> kf, Win<float> wf, const PbGeo *geo, const double *selfblk,
                              const int32_t *boff, const int64_t *belem, const int64_t *moff, int nc, int sys,
                              float *M) {
    int b = blockIdx.y;
    int m = boff[b + 1] - boff[b];
    int64_t pair = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pair >= (int64_t)m * m) return;
    int i = (int)(pair / m), j = (int)(pair % m);
    int64_t ei = belem[boff[b] + i], ej = belem[boff[b] + j];
    float o[3][3];
    if (ei == ej) {
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) o[r][c] = (float)selfblk[9 * ei + 3 * r + c];
    } else {
        pair_block(kf, wf, geo[ei], geo[ej], o);
    }
    if (sys == DDM_SYS_RATE)
        for (int c = 0; c < 3; ++c) o[1][c] += o[2][c];
    int n = nc * m;
    float *A = M + moff[b];
    for (int rc = 0; rc < nc; ++rc)
        for (int cc = 0; cc < nc; ++cc) A[(int64_t)(rc * m + i) * n + cc * m + j] = o[rc][cc];
}

// In-place Gauss-Jordan inversion with partial pivoting, one CTA per
// matrix (n <= 192) held in registers: 32 x 32 threads, thread (tx, ty)
// owns rows ty + 32 i and columns tx + 32 j (i, j < 6).  Step k:
//   1. the owners of column k post their best pivot candidate; every warp
//      reduces the 32 candidates itself (same result everywhere);
//   2. the pivot row (pre-swap row pr), the old row k and column k go to
//      shared memory;
//   3. every thread updates its entries; the swap is folded in: row k takes
//      the scaled pivot row, row pr takes the old row k, and the column-k
//      multipliers of rows k and pr are exchanged.
// The band of 32 columns (i = k / 32) is a compile-time index (unrolled
// outer loop), so the pivot column lives in fixed registers.
constexpr int INV_MAX = 3 * 64, GJ_R = INV_MAX / 32;
__global__ void __launch_bounds__(1024, 1) k_pb_invert(const int32_t *boff, const int64_t *moff, int nc, float *M) {
    __shared__ float prow[INV_MAX], orow[INV_MAX], colk[INV_MAX], cand_v[32];
    __shared__ int piv[INV_MAX], cand_r[32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int b = blockIdx.x;
    const int n = nc * (boff[b + 1] - boff[b]);
    float *G = M + moff[b];
    float a[GJ_R][GJ_R];
#pragma unroll
    for (int i = 0; i < GJ_R; ++i)
#pragma unroll
        for (int j = 0; j < GJ_R; ++j) {
            const int r = ty + 32 * i, c = tx + 32 * j;
            a[i][j] = (r < n && c < n) ? G[r * n + c] : 0.f;
        }
#pragma unroll
    for (int ki = 0; ki < GJ_R; ++ki) {
        for (int kt = 0; kt < 32; ++kt) {
            const int k = 32 * ki + kt;
            if (k >= n) break;
            // 1. pivot candidates of the column-k owners, reduced by every warp
            if (tx == kt) {
                float best = -1.f;
                int bi = k;
#pragma unroll
                for (int i = 0; i < GJ_R; ++i) {
                    const int r = ty + 32 * i;
                    if (r >= k && r < n && fabsf(a[i][ki]) > best) { best = fabsf(a[i][ki]); bi = r; }
                }
                cand_v[ty] = best;
                cand_r[ty] = bi;
            }
            __syncthreads();
            float pv = cand_v[tx];
            int pr = cand_r[tx];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xFFFFFFFFu, pv, o);
                const int orr = __shfl_xor_sync(0xFFFFFFFFu, pr, o);
                if (ov > pv || (ov == pv && orr < pr)) { pv = ov; pr = orr; }
            }
            if (tx == 0 && ty == 0) piv[k] = pr;
            const int pi = pr >> 5, pt = pr & 31;
            // 2. pivot row, old row k, column k
            if (ty == pt)
#pragma unroll
                for (int i = 0; i < GJ_R; ++i)
                    if (i == pi)
#pragma unroll
                        for (int j = 0; j < GJ_R; ++j) prow[tx + 32 * j] = a[i][j];
            if (ty == kt && pr != k)
#pragma unroll
                for (int j = 0; j < GJ_R; ++j) orow[tx + 32 * j] = a[ki][j];
            if (tx == kt)
#pragma unroll
                for (int i = 0; i < GJ_R; ++i) colk[ty + 32 * i] = a[i][ki];
            __syncthreads();
            // 3. update: one FMA per entry, then the rows k and pr and the
            //    column k are overwritten (row k <- scaled pivot row, row pr
            //    <- old row k eliminated, column k <- -multiplier / pivot)
            const float p = prow[k];
            const float ip = p != 0.f ? 1.f / p : 0.f;
            float pc[GJ_R], m[GJ_R];
#pragma unroll
            for (int j = 0; j < GJ_R; ++j) pc[j] = prow[tx + 32 * j] * ip;
#pragma unroll
            for (int i = 0; i < GJ_R; ++i) m[i] = colk[ty + 32 * i];
#pragma unroll
            for (int i = 0; i < GJ_R; ++i)
#pragma unroll
                for (int j = 0; j < GJ_R; ++j) a[i][j] = fmaf(-m[i], pc[j], a[i][j]);
            if (ty == pt && pr != k) {            // row pr: the old row k, eliminated
                const float mp = colk[k];
#pragma unroll
                for (int i = 0; i < GJ_R; ++i)
                    if (i == pi) {
                        m[i] = mp;
#pragma unroll
                        for (int j = 0; j < GJ_R; ++j) a[i][j] = fmaf(-mp, pc[j], orow[tx + 32 * j]);
                    }
            }
            if (tx == kt)                         // column k
#pragma unroll
                for (int i = 0; i < GJ_R; ++i) a[i][ki] = -m[i] * ip;
            if (ty == kt) {                       // row k (and the pivot position)
#pragma unroll
                for (int j = 0; j < GJ_R; ++j) a[ki][j] = pc[j];
                if (tx == kt) a[ki][ki] = ip;
            }
            __syncthreads();                  // shared rows are rewritten by the next step
        }
    }
    // undo the row interchanges as column swaps, in reverse order (a warp
    // holds whole rows: shuffles)
    for (int k = n - 1; k >= 0; --k) {
        const int pr = piv[k];
        if (pr == k) continue;
        const int kj = k >> 5, kt = k & 31, pj = pr >> 5, pt = pr & 31;
#pragma unroll
        for (int i = 0; i < GJ_R; ++i) {
            float vk = 0.f, vp = 0.f;
#pragma unroll
            for (int j = 0; j < GJ_R; ++j) {
                if (j == kj) vk = a[i][j];
                if (j == pj) vp = a[i][j];
            }
            vk = __shfl_sync(0xFFFFFFFFu, vk, kt);
            vp = __shfl_sync(0xFFFFFFFFu, vp, pt);
#pragma unroll
            for (int j = 0; j < GJ_R; ++j) {
                if (tx == kt && j == kj) a[i][j] = vp;
                if (tx == pt && j == pj) a[i][j] = vk;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < GJ_R; ++i)
#pragma unroll
        for (int j = 0; j < GJ_R; ++j) {
            const int r = ty + 32 * i, c = tx + 32 * j;
            if (r < n && c < n) G[r * n + c] = a[i][j];
        }
}

// z (3N layout, caller order) = Minv v (v in the system layout nc x N);
// PA_S CTAs per chain block, each a slice of its rows; a warp takes PA_R rows
// at a time, lanes along the rows (coalesced); the unknown blocks beyond nc
// are set to zero
constexpr int PA_T = 256, PA_WARPS = PA_T / 32, PA_R = 4, PA_S = 2;
__device__ __forceinline__ void pb_apply_body(const int32_t *boff, const int64_t *belem, const int64_t *moff, int nc,
                                              const float *Minv, const double *v, int64_t N, double *z,
                                              int zero_rest, int b) {
    __shared__ float sv[INV_MAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = boff[b + 1] - boff[b], n = nc * m;
    const int64_t *el = belem + boff[b];
    for (int c = threadIdx.x; c < n; c += PA_T) sv[c] = (float)v[(c / m) * N + el[c % m]];
    __syncthreads();
    const float *A = Minv + moff[b];
    // this CTA's rows: slice blockIdx.y of PA_S; PA_R rows per warp step, all
    // their loads issued before the first multiply
    const int rs = (n + PA_S - 1) / PA_S, r0 = blockIdx.y * rs, r1 = min(n, r0 + rs);
    for (int rb = r0 + PA_R * warp; rb < r1; rb += PA_R * PA_WARPS) {
        float s[PA_R];
        const float *Ar[PA_R];
#pragma unroll
        for (int q = 0; q < PA_R; ++q) {
            s[q] = 0.f;
            Ar[q] = A + (int64_t)min(rb + q, r1 - 1) * n;
        }
        // n <= INV_MAX: every load of the PA_R rows is issued up front
        float a[INV_MAX / 32][PA_R];
#pragma unroll
        for (int k = 0; k < INV_MAX / 32; ++k) {
            const int c = lane + 32 * k;
#pragma unroll
            for (int q = 0; q < PA_R; ++q) a[k][q] = c < n ? Ar[q][c] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < INV_MAX / 32; ++k) {
            const int c = lane + 32 * k;
            const float x = c < n ? sv[c] : 0.f;
#pragma unroll
            for (int q = 0; q < PA_R; ++q) s[q] = fmaf(a[k][q], x, s[q]);
        }
#pragma unroll
        for (int q = 0; q < PA_R; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xFFFFFFFFu, s[q], o);
#pragma unroll
        for (int q = 0; q < PA_R; ++q) {
            const int r = rb + q;
            if (lane == q && r < r1) z[(r / m) * N + el[r % m]] = (double)s[q];
        }
    }
    if (zero_rest && nc < 3 && blockIdx.y == 0)
        for (int e = threadIdx.x; e < m; e += PA_T) z[2 * N + el[e]] = 0.0;
}
__global__ void __launch_bounds__(PA_T) k_pb_apply(const int32_t *boff, const int64_t *belem, const int64_t *moff,
                                                   int nc, const float *Minv, const double *v, int64_t N, double *z,
                                                   int zero_rest) {
    pb_apply_body(boff, belem, moff, nc, Minv, v, N, z, zero_rest, blockIdx.x);
}

// ------------------------------------------------------------ coarse level
// Legendre polynomial P_k (k < 3) at the centre of element i of an m-element
// block, mapped to [-1, 1]
__device__ __forceinline__ float leg(int k, int i, int m) {
    const float t = -1.f + (2.f * i + 1.f) / (float)m;
    return k == 0 ? 1.f : (k == 1 ? t : 1.5f * t * t - 0.5f);
}
constexpr int PC_T = 128, PC_MAXQ = 3 * PC_MODES;
// A_c[(I nc + c) K + k][(J nc + d) K + l] = sum_{i in I, j in J}
//     P_k(t_i) A_{(c, i), (d, j)} P_l(t_j): one CTA per (coarse block I,
// coarse block J), the element pairs split over the threads
__global__ void __launch_bounds__(PC_T) k_pc_assemble(KConst<float> kf, Win<float> wf, const PbGeo *geo,
                                                      const double *selfblk, const int32_t *boff,
                                                      const int64_t *belem, const int32_t *pcb, int nc, int sys,
                                                      int K, int64_t dim, float *Ac) {
    __shared__ float red[PC_T / 32][PC_MAXQ * PC_MAXQ];
    const int I = blockIdx.x, J = blockIdx.y;
    const int bI = pcb[I], bJ = pcb[J];
    const int mI = boff[bI + 1] - boff[bI], mJ = boff[bJ + 1] - boff[bJ];
    const int64_t *elI = belem + boff[bI], *elJ = belem + boff[bJ];
    const int Q = nc * K;
    float acc[PC_MAXQ][PC_MAXQ];
#pragma unroll
    for (int a = 0; a < PC_MAXQ; ++a)
#pragma unroll
        for (int b = 0; b < PC_MAXQ; ++b) acc[a][b] = 0.f;
    for (int p = threadIdx.x; p < mI * mJ; p += PC_T) {
        const int i = p / mJ, j = p % mJ;
        const int64_t ei = elI[i], ej = elJ[j];
        float o[3][3];
        if (ei == ej) {
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) o[r][c] = (float)selfblk[9 * ei + 3 * r + c];
        } else {
            pair_block(kf, wf, geo[ei], geo[ej], o);
        }
        if (sys == DDM_SYS_RATE)
            for (int c = 0; c < 3; ++c) o[1][c] += o[2][c];
        float pi[PC_MODES], pj[PC_MODES];
#pragma unroll
        for (int k = 0; k < PC_MODES; ++k) { pi[k] = leg(k, i, mI); pj[k] = leg(k, j, mJ); }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < PC_MODES; ++k)
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int l = 0; l < PC_MODES; ++l)
                        if (c < nc && d < nc && k < K && l < K)
                            acc[c * PC_MODES + k][d * PC_MODES + l] =
                                fmaf(o[c][d] * pi[k], pj[l], acc[c * PC_MODES + k][d * PC_MODES + l]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < PC_MAXQ; ++a)
#pragma unroll
        for (int b = 0; b < PC_MAXQ; ++b) {
            float v = acc[a][b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            if (lane == 0) red[warp][a * PC_MAXQ + b] = v;
        }
    __syncthreads();
    for (int q = threadIdx.x; q < Q * Q; q += PC_T) {
        const int a = q / Q, b = q % Q;              // a = c K + k, b = d K + l
        const int c = a / K, k = a % K, d = b / K, l = b % K;
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < PC_T / 32; ++w) v += red[w][(c * PC_MODES + k) * PC_MAXQ + d * PC_MODES + l];
        Ac[((int64_t)I * Q + a) * dim + (int64_t)J * Q + b] = v;
    }
}

// In-place Gauss-Jordan inversion of the coarse matrices (FP32, partial
// pivoting).  For one step k the pivot kernel swaps the pivot row into
// place and stages row k (scaled by 1/pivot) and column k; the update
// kernel then rewrites every entry from the staged copies, so that no entry
// is read after it was overwritten.
constexpr int GJ_T = 1024;
// The same steps for many coarse matrices at once: at step k the problems
// whose dimension exceeds k (a prefix: they are sorted by dimension,
// largest first) take part; one CTA per problem stages its pivot row and
// column, then one flat grid over all their entries updates them.
struct GjDesc {
    float *A;          // dim x dim, row-major
    float *stage;      // 2 dim + 1: row k / pivot, column k, 1 / pivot
    int32_t *piv;
    int64_t dim;
};
__global__ void __launch_bounds__(GJ_T) k_gjb_pivot(const GjDesc *D, int64_t k) {
    const GjDesc d = D[blockIdx.x];
    float *A = d.A;
    const int64_t n = d.dim;
    __shared__ float bv[GJ_T / 32];
    __shared__ int64_t bi[GJ_T / 32];
    __shared__ int64_t s_p;
    float best = -1.f;
    int64_t bidx = k;
    for (int64_t i = k + threadIdx.x; i < n; i += GJ_T) {
        const float v = fabsf(A[i * n + k]);
        if (v > best) { best = v; bidx = i; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        const int64_t oi = __shfl_xor_sync(0xFFFFFFFFu, bidx, o);
        if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if (lane == 0) { bv[warp] = best; bi[warp] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = bv[0];
        int64_t p = bi[0];
        for (int w = 1; w < GJ_T / 32; ++w)
            if (bv[w] > b || (bv[w] == b && bi[w] < p)) { b = bv[w]; p = bi[w]; }
        s_p = p;
        d.piv[k] = (int32_t)p;
    }
    __syncthreads();
    const int64_t p = s_p;
    if (p != k)
        for (int64_t j = threadIdx.x; j < n; j += GJ_T) {
            const float a = A[k * n + j];
            A[k * n + j] = A[p * n + j];
            A[p * n + j] = a;
        }
    __syncthreads();
    const float pv = A[k * n + k];
    const float ip = pv != 0.f ? 1.f / pv : 0.f;
    for (int64_t j = threadIdx.x; j < n; j += GJ_T) {
        d.stage[j] = A[k * n + j] * ip;
        d.stage[n + j] = A[j * n + k];
    }
    if (threadIdx.x == 0) d.stage[2 * n] = ip;
}
constexpr int GJB_CH = 2048;          // entries per CTA of the update
__global__ void __launch_bounds__(256) k_gjb_update(const GjDesc *D, const int64_t *cum, int m, int64_t k) {
    // the CTA's problem: first p with cum[p + 1] > blockIdx.x (cum[0] = 0)
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cum[mid + 1] > (int64_t)blockIdx.x) hi = mid; else lo = mid + 1;
    }
    const GjDesc d = D[lo];
    const int64_t n = d.dim, base = ((int64_t)blockIdx.x - cum[lo]) * GJB_CH;
    const float ip = d.stage[2 * n];
    for (int64_t q = base + threadIdx.x; q < base + GJB_CH && q < n * n; q += 256) {
        const int64_t i = q / n, j = q % n;
        float v;
        if (i == k) v = j == k ? ip : d.stage[j];
        else v = j == k ? -d.stage[n + i] * ip : fmaf(-d.stage[n + i], d.stage[j], d.A[q]);
        d.A[q] = v;
    }
}
// column swaps of every problem, a thread per row (grid.y = problem)
__global__ void k_gjb_unpivot(const GjDesc *D) {
    const GjDesc d = D[blockIdx.y];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= d.dim) return;
    float *row = d.A + i * d.dim;
    for (int64_t k = d.dim - 1; k >= 0; --k) {
        const int64_t p = d.piv[k];
        if (p != k) { const float a = row[k]; row[k] = row[p]; row[p] = a; }
    }
}

// coarse residual r_c = Z^T v (FP64 sums), one CTA per coarse block
__global__ void k_pc_restrict(const double *v, int64_t N, const int32_t *boff, const int64_t *belem,
                              const int32_t *pcb, int nc, int K, float *rc) {
    __shared__ double red[2][PC_MAXQ];
    const int I = blockIdx.x, b = pcb[I], m = boff[b + 1] - boff[b];
    const int64_t *el = belem + boff[b];
    double acc[PC_MAXQ];
#pragma unroll
    for (int q = 0; q < PC_MAXQ; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < m; i += 64)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (c < nc) {
                const double x = v[c * N + el[i]];
#pragma unroll
                for (int k = 0; k < PC_MODES; ++k)
                    if (k < K) acc[c * PC_MODES + k] += (double)leg(k, i, m) * x;
            }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < PC_MAXQ; ++q) {
        double a = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        if (lane == 0) red[warp][q] = a;
    }
    __syncthreads();
    const int Q = nc * K;
    if (threadIdx.x < Q) {
        const int c = threadIdx.x / K, k = threadIdx.x % K;
        rc[(int64_t)I * Q + threadIdx.x] = (float)(red[0][c * PC_MODES + k] + red[1][c * PC_MODES + k]);
    }
}
// y_c = A_c^-1 r_c, a warp per row
__global__ void k_pc_gemv(const float *Ainv, const float *rc, int64_t n, float *yc) {
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *row = Ainv + r * n;
    float s = 0.f;
    for (int64_t j = lane; j < n; j += 32) s = fmaf(row[j], rc[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) yc[r] = s;
}
// z += Z y_c
__global__ void k_pc_prolong(const float *yc, int64_t N, const int32_t *boff, const int64_t *belem,
                             const int32_t *pcb, int nc, int K, double *z) {
    const int I = blockIdx.x, b = pcb[I], m = boff[b + 1] - boff[b];
    const int64_t *el = belem + boff[b];
    const int Q = nc * K;
    for (int i = threadIdx.x; i < m; i += 64)
        for (int c = 0; c < nc; ++c) {
            float s = 0.f;
            for (int k = 0; k < K; ++k) s = fmaf(leg(k, i, m), yc[(int64_t)I * Q + c * K + k], s);
            z[c * N + el[i]] += (double)s;
        }
}

// ---- batched apply: every problem of a batch in one launch per stage
struct PbDesc {
    const int32_t *boff, *pcb;
    const int64_t *belem, *moff;
    const float *Minv, *Ainv;
    float *rc, *yc;
    const double *v;
    double *z;
    int64_t N, dim;
    int K;
};
// one CTA per (problem, block) x row slice
// act (may be null): problems whose flag is 0 are skipped
__global__ void __launch_bounds__(PA_T) k_pb_apply_b(const PbDesc *D, const int2 *items, int nc, const int *act) {
    const int2 w = items[blockIdx.x];
    if (act && !act[w.x]) return;
    const PbDesc &d = D[w.x];
    pb_apply_body(d.boff, d.belem, d.moff, nc, d.Minv, d.v, d.N, d.z, 1, w.y);
}
// items (p, coarse block I)
__global__ void k_pc_restrict_b(const PbDesc *D, const int2 *items, int nc, const int *act) {
    const int2 w = items[blockIdx.x];
    if (act && !act[w.x]) return;
    const PbDesc &d = D[w.x];
    __shared__ double red[2][PC_MAXQ];
    const int I = w.y, b = d.pcb[I], m = d.boff[b + 1] - d.boff[b], K = d.K;
    const int64_t *el = d.belem + d.boff[b];
    double acc[PC_MAXQ];
#pragma unroll
    for (int q = 0; q < PC_MAXQ; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < m; i += 64)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (c < nc) {
                const double x = d.v[c * d.N + el[i]];
#pragma unroll
                for (int k = 0; k < PC_MODES; ++k)
                    if (k < K) acc[c * PC_MODES + k] += (double)leg(k, i, m) * x;
            }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < PC_MAXQ; ++q) {
        double a = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        if (lane == 0) red[warp][q] = a;
    }
    __syncthreads();
    const int Q = nc * K;
    if (threadIdx.x < Q) {
        const int c = threadIdx.x / K, k = threadIdx.x % K;
        d.rc[(int64_t)I * Q + threadIdx.x] = (float)(red[0][c * PC_MODES + k] + red[1][c * PC_MODES + k]);
    }
}
// items (p, first of 8 rows); a warp per row
__global__ void k_pc_gemv_b(const PbDesc *D, const int2 *items, const int *act) {
    const int2 w = items[blockIdx.x];
    if (act && !act[w.x]) return;
    const PbDesc &d = D[w.x];
    const int64_t r = (int64_t)w.y + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= d.dim) return;
    const float *row = d.Ainv + r * d.dim;
    float sacc = 0.f;
    for (int64_t j = lane; j < d.dim; j += 32) sacc = fmaf(row[j], d.rc[j], sacc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xFFFFFFFFu, sacc, o);
    if (lane == 0) d.yc[r] = sacc;
}
__global__ void k_pc_prolong_b(const PbDesc *D, const int2 *items, int nc, const int *act) {
    const int2 w = items[blockIdx.x];
    if (act && !act[w.x]) return;
    const PbDesc &d = D[w.x];
    const int I = w.y, b = d.pcb[I], m = d.boff[b + 1] - d.boff[b], K = d.K;
    const int64_t *el = d.belem + d.boff[b];
    const int Q = nc * K;
    for (int i = threadIdx.x; i < m; i += 64)
        for (int c = 0; c < nc; ++c) {
            float sacc = 0.f;
            for (int k = 0; k < K; ++k) sacc = fmaf(leg(k, i, m), d.yc[(int64_t)I * Q + c * K + k], sacc);
            d.z[c * d.N + el[i]] += (double)sacc;
        }
}

}  // namespace

struct BatchPb {
    int np = 0, nc = 0;
    const int *act = nullptr;
    PbDesc *desc = nullptr;
    int2 *blk = nullptr, *pc = nullptr, *gemv = nullptr;
    int n_blk = 0, n_pc = 0, n_gemv = 0;
};

void bpb_free(BatchPb *b, cudaStream_t s) {
    if (!b) return;
    void *ps[] = {b->desc, b->blk, b->pc, b->gemv};
    for (void *p : ps) dfree(p, s);
    delete b;
}

// the batched preconditioner of problems p (prepared for the same (dt,
// system)) from v_p (system layout) into z_p (3N layout)
ddm_status bpb_build(ddm_ctx *ctx, ddm_tree *const *trees, int np, int sys, const double *const *vs,
                     double *const *zs, const int *act, cudaStream_t s, BatchPb **out) {
    *out = nullptr;
    const int nc = sys == DDM_SYS_PRESSURE ? 3 : 2;
    std::vector<PbDesc> hd(np);
    std::vector<int2> hblk, hpc, hgemv;
    for (int p = 0; p < np; ++p) {
        ddm_tree *t = trees[p];
        if (!t->pb_inv || t->pb_sys != sys) return ctx_fail(ctx, DDM_EINVAL, "batched preconditioner: not prepared");
        PbDesc &d = hd[p];
        d.boff = t->pb_off; d.belem = t->pb_elem; d.moff = t->pb_moff; d.Minv = t->pb_inv;
        d.v = vs[p]; d.z = zs[p]; d.N = t->n;
        d.pcb = t->pc_blk; d.K = t->pc_modes; d.Ainv = t->pc_inv; d.dim = 0; d.rc = d.yc = nullptr;
        for (int64_t b = 0; b < t->n_pblk; ++b) hblk.push_back(make_int2(p, (int)b));
        if (t->n_pc > 0) {
            const int K = t->pc_modes;
            d.dim = t->n_pc * nc * K;
            d.rc = t->pc_inv + (size_t)t->n_pc * 3 * K * t->n_pc * 3 * K;
            d.yc = d.rc + t->n_pc * 3 * K;
            for (int64_t I = 0; I < t->n_pc; ++I) hpc.push_back(make_int2(p, (int)I));
            for (int64_t r = 0; r < d.dim; r += 8) hgemv.push_back(make_int2(p, (int)r));
        }
    }
    BatchPb *b = new BatchPb();
    b->np = np; b->nc = nc; b->act = act;
    b->n_blk = (int)hblk.size(); b->n_pc = (int)hpc.size(); b->n_gemv = (int)hgemv.size();
    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        if (dalloc(dst, bytes ? bytes : 16, s) != cudaSuccess) return false;
        return !bytes || cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    bool ok = up((void **)&b->desc, hd.data(), hd.size() * sizeof(PbDesc)) &&
              up((void **)&b->blk, hblk.data(), hblk.size() * sizeof(int2)) &&
              up((void **)&b->pc, hpc.data(), hpc.size() * sizeof(int2)) &&
              up((void **)&b->gemv, hgemv.data(), hgemv.size() * sizeof(int2)) &&
              cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        bpb_free(b, s);
        return ctx_fail(ctx, DDM_ENOMEM, "batched preconditioner: work list allocation failed");
    }
    *out = b;
    return DDM_OK;
}

ddm_status bpb_launch(ddm_ctx *ctx, BatchPb *b, cudaStream_t s) {
    int launches = 0;
    if (b->n_blk > 0) {
        k_pb_apply_b<<<dim3((unsigned)b->n_blk, PA_S), PA_T, 0, s>>>(b->desc, b->blk, b->nc, b->act);
        ++launches;
    }
    if (b->n_pc > 0) {
        k_pc_restrict_b<<<(unsigned)b->n_pc, 64, 0, s>>>(b->desc, b->pc, b->nc, b->act);
        k_pc_gemv_b<<<(unsigned)b->n_gemv, 256, 0, s>>>(b->desc, b->gemv, b->act);
        k_pc_prolong_b<<<(unsigned)b->n_pc, 64, 0, s>>>(b->desc, b->pc, b->nc, b->act);
        launches += 3;
    }
    prof_end(ctx, 8, launches);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

// invert the pending coarse matrices of the given trees together (batched
// Gauss-Jordan: 2 max_dim + 1 launches for all of them)
ddm_status pc_invert_many(ddm_ctx *ctx, ddm_tree *const *trees, int count, cudaStream_t s) {
    std::vector<ddm_tree *> pend;
    for (int i = 0; i < count; ++i)
        if (trees[i]->n_pc > 0 && trees[i]->pc_pending) pend.push_back(trees[i]);
    if (pend.empty()) return DDM_OK;
    auto dim_of = [](const ddm_tree *t) { return t->n_pc * (t->pb_sys == DDM_SYS_PRESSURE ? 3 : 2) * t->pc_modes; };
    std::sort(pend.begin(), pend.end(), [&](const ddm_tree *a, const ddm_tree *b) { return dim_of(a) > dim_of(b); });
    const int P = (int)pend.size();
    std::vector<GjDesc> hd(P);
    std::vector<int64_t> dims(P), cum(P + 1, 0);
    int64_t scratch = 0;
    for (int p = 0; p < P; ++p) {
        dims[p] = dim_of(pend[p]);
        scratch += 2 * dims[p] + 1;
    }
    float *stage = nullptr;
    int32_t *piv = nullptr;
    GjDesc *dd = nullptr;
    int64_t *dcum = nullptr;
    int64_t tot_piv = 0;
    for (int p = 0; p < P; ++p) tot_piv += dims[p];
    DDM_CUDA_TRY(ctx, dalloc(&stage, (size_t)scratch * sizeof(float), s));
    DDM_CUDA_TRY(ctx, dalloc(&piv, (size_t)tot_piv * sizeof(int32_t), s));
    DDM_CUDA_TRY(ctx, dalloc(&dd, (size_t)P * sizeof(GjDesc), s));
    DDM_CUDA_TRY(ctx, dalloc(&dcum, (size_t)(P + 1) * sizeof(int64_t), s));
    int64_t so = 0, po = 0;
    for (int p = 0; p < P; ++p) {
        hd[p] = GjDesc{pend[p]->pc_inv, stage + so, piv + po, dims[p]};
        so += 2 * dims[p] + 1;
        po += dims[p];
        cum[p + 1] = cum[p] + (dims[p] * dims[p] + GJB_CH - 1) / GJB_CH;
    }
    DDM_CUDA_TRY(ctx, cudaMemcpyAsync(dd, hd.data(), P * sizeof(GjDesc), cudaMemcpyHostToDevice, s));
    DDM_CUDA_TRY(ctx, cudaMemcpyAsync(dcum, cum.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    prof_begin(ctx, 8);
    const int64_t maxd = dims[0];
    int m = P;
    for (int64_t k = 0; k < maxd; ++k) {
        while (m > 0 && dims[m - 1] <= k) --m;          // problems still eliminating
        k_gjb_pivot<<<m, GJ_T, 0, s>>>(dd, k);
        k_gjb_update<<<(unsigned)cum[m], 256, 0, s>>>(dd, dcum, m, k);
    }
    k_gjb_unpivot<<<dim3((unsigned)((maxd + 255) / 256), (unsigned)P), 256, 0, s>>>(dd);
    prof_end(ctx, 8, (int)(2 * maxd + 1));
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));    // host descriptor vectors go out of scope
    dfree(stage, s);
    dfree(piv, s);
    dfree(dd, s);
    dfree(dcum, s);
    for (ddm_tree *t : pend) t->pc_pending = false;
    return DDM_OK;
}

// prepare the inverted blocks of (dt, system) for tree t (cached); with
// defer_coarse the coarse matrix is assembled and left for pc_invert_many
ddm_status pb_prepare(ddm_ctx *ctx, ddm_tree *t, double dt, int sys, cudaStream_t s, bool defer_coarse) {
    if (t->pb_inv && t->pb_dt == dt && t->pb_sys == sys) return DDM_OK;
    int nc = sys == DDM_SYS_PRESSURE ? 3 : 2;
    if (!t->pb_inv) DDM_CUDA_TRY(ctx, dalloc(&t->pb_inv, std::max<int64_t>(t->pb_msize, 1) * sizeof(float), t->stream));
    // the matrices of a 2N system are packed into the same per-block slots
    Win<double> w;
    w.ct_hi = ctx->kd.c * dt;
    w.ct_lo = 0.0;
    w.g_hi = 1.0 / (4.0 * ctx->kd.c * dt);
    w.g_lo = 0.0;
    w.elastic = 1;
    Win<float> wf{(float)w.ct_hi, 0.f, (float)w.g_hi, 0.f, 1};
    const double *selfblk = nullptr;                // own elements (window (0, dt)), FP64, cached
    ddm_status st = window_self_blocks(ctx, t, 0.0, dt, s, &selfblk);
    if (st) return st;
    PbGeo *geo = nullptr;
    DDM_CUDA_TRY(ctx, dalloc(&geo, (size_t)t->n * sizeof(PbGeo), s));
    prof_begin(ctx, 8);
    k_pb_geom<<<(unsigned)((t->n + 255) / 256), 256, 0, s>>>(t->xy_caller, t->n, geo);
    int64_t mm = (int64_t)t->pb_max * t->pb_max;
    dim3 g((unsigned)((mm + 127) / 128), (unsigned)t->n_pblk);
    k_pb_assemble<<<g, 128, 0, s>>>(ctx->kf, wf, geo, selfblk, t->pb_off, t->pb_elem, t->pb_moff, nc, sys,
                                    t->pb_inv);
    k_pb_invert<<<(unsigned)t->n_pblk, dim3(32, 32), 0, s>>>(t->pb_off, t->pb_moff, nc, t->pb_inv);
    prof_end(ctx, 8, 4);
    if (t->n_pc > 0) {
        // coarse level: Galerkin matrix of the long chains' blocks, inverted
        const int K = t->pc_modes;
        const int64_t dim = t->n_pc * nc * K;
        if (!t->pc_inv)
            DDM_CUDA_TRY(ctx, dalloc(&t->pc_inv, ((size_t)t->n_pc * 3 * K * t->n_pc * 3 * K + 2 * t->n_pc * 3 * K) *
                                                     sizeof(float), t->stream));
        prof_begin(ctx, 8);
        k_pc_assemble<<<dim3((unsigned)t->n_pc, (unsigned)t->n_pc), PC_T, 0, s>>>(
            ctx->kf, wf, geo, selfblk, t->pb_off, t->pb_elem, t->pc_blk, nc, sys, K, dim, t->pc_inv);
        prof_end(ctx, 8, 1);
        t->pc_pending = true;
    }
    dfree(geo, s);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    t->pb_dt = dt;
    t->pb_sys = sys;
    if (t->n_pc > 0 && !defer_coarse) return pc_invert_many(ctx, &t, 1, s);
    return DDM_OK;
}

// z = M^-1 v : v in the system layout (nc blocks of N), z in the 3N layout
ddm_status pb_apply(ddm_ctx *ctx, ddm_tree *t, int sys, const double *v, double *z, cudaStream_t s) {
    int nc = sys == DDM_SYS_PRESSURE ? 3 : 2;
    k_pb_apply<<<dim3((unsigned)t->n_pblk, PA_S), PA_T, 0, s>>>(t->pb_off, t->pb_elem, t->pb_moff, nc, t->pb_inv, v, t->n, z, 1);
    prof_end(ctx, 8, 1);
    if (t->n_pc > 0) {             // + Z A_c^-1 Z^T v
        const int K = t->pc_modes;
        const int64_t dim = t->n_pc * nc * K;
        float *rc = t->pc_inv + (size_t)t->n_pc * 3 * K * t->n_pc * 3 * K, *yc = rc + t->n_pc * 3 * K;
        k_pc_restrict<<<(unsigned)t->n_pc, 64, 0, s>>>(v, t->n, t->pb_off, t->pb_elem, t->pc_blk, nc, K, rc);
        k_pc_gemv<<<(unsigned)((dim + 7) / 8), 256, 0, s>>>(t->pc_inv, rc, dim, yc);
        k_pc_prolong<<<(unsigned)t->n_pc, 64, 0, s>>>(yc, t->n, t->pb_off, t->pb_elem, t->pc_blk, nc, K, z);
        prof_end(ctx, 8, 3);
    }
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}
