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
__global__ void __launch_bounds__(PA_T) k_pb_apply(const int32_t *boff, const int64_t *belem, const int64_t *moff,
                                                   int nc, const float *Minv, const double *v, int64_t N, double *z,
                                                   int zero_rest) {
    __shared__ float sv[INV_MAX];
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

}  // namespace

// prepare the inverted blocks of (dt, system) for tree t (cached)
ddm_status pb_prepare(ddm_ctx *ctx, ddm_tree *t, double dt, int sys, cudaStream_t s) {
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
    dfree(geo, s);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    t->pb_dt = dt;
    t->pb_sys = sys;
    return DDM_OK;
}

// z = M^-1 v : v in the system layout (nc blocks of N), z in the 3N layout
ddm_status pb_apply(ddm_ctx *ctx, ddm_tree *t, int sys, const double *v, double *z, cudaStream_t s) {
    int nc = sys == DDM_SYS_PRESSURE ? 3 : 2;
    k_pb_apply<<<dim3((unsigned)t->n_pblk, PA_S), PA_T, 0, s>>>(t->pb_off, t->pb_elem, t->pb_moff, nc, t->pb_inv, v, t->n, z, 1);
    prof_end(ctx, 8, 1);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}
