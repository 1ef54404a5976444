// Block-Jacobi preconditioner over fracture chains.
//
// Elements that share end points form chains (one fracture); the chains are
// cut into blocks of at most 64 elements at tree build.  For a time step dt
// each block's own influence matrix (all its element pairs: FP32 closed
// forms for the DD part on FP64 offsets, Gauss rule for the fluid source,
// the own element in FP64 closed form) is assembled for the rows and
// unknowns of the system being solved and inverted on the device in FP32
// (Gauss-Jordan with partial pivoting, one thread block per matrix); a
// preconditioner needs no more precision, and FP32 runs at 64x the FP64
// rate of this part.  Applying the preconditioner is
// one small dense product per block.  Elements that belong to no chain form
// 1-element blocks, i.e. the own-element 3x3 block Jacobi.
#include <cmath>
#include <vector>

#include "internal.h"
#include "kernel_math.cuh"

namespace {

constexpr int PT = 256;

// Gauss-Legendre, 8 points on [-1, 1] (fluid source between elements)
__constant__ double c_gl8x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                                 0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
__constant__ double c_gl8w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                                 0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

// rows (sigma_s, sigma_n, p) at element i's midpoint from unit (Ds, Dn, Dq)
// on element j: FP32 pair arithmetic on offsets taken in FP64 (the
// preconditioner needs no more), own element in FP64 closed form
__device__ void pair_block(const KConst<float> &kf, const Win<float> &wf, const KConst<double> &kd,
                           const Win<double> &wd, const double *xy, int64_t N, int64_t i, int64_t j, float out[3][3]) {
    double ax = xy[i], ay = xy[N + i], bx = xy[2 * N + i], by = xy[3 * N + i];
    double Li = hypot(bx - ax, by - ay), tix = (bx - ax) / Li, tiy = (by - ay) / Li;
    if (i == j) {
        for (int c = 0; c < 3; ++c) {
            double o[3];
            self_field(kd, wd, 0.5 * Li, tix, tiy, c == 0, c == 1, c == 2, o);
            for (int r = 0; r < 3; ++r) out[r][c] = (float)o[r];
        }
        return;
    }
    double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
    double cx = xy[j], cy = xy[N + j], dx = xy[2 * N + j], dy = xy[3 * N + j];
    double Lj = hypot(dx - cx, dy - cy);
    float tjx = (float)((dx - cx) / Lj), tjy = (float)((dy - cy) / Lj), njx = -tjy, njy = tjx;
    float z1x = (float)(mx - cx), z1y = (float)(my - cy), z2x = (float)(mx - dx), z2y = (float)(my - dy);
    float ftx = (float)tix, fty = (float)tiy;
    for (int c = 0; c < 2; ++c) {
        float Dx = c == 0 ? tjx : njx, Dy = c == 0 ? tjy : njy;
        float g[4] = {0, 0, 0, 0};
        disl_field<float>(kf, z1x, z1y, Dx, Dy, wf, 1.f, g);
        disl_field<float>(kf, z2x, z2y, Dx, Dy, wf, -1.f, g);
        float ss, sn;
        to_local<float>(ftx, fty, g, ss, sn);
        out[0][c] = ss; out[1][c] = sn; out[2][c] = g[3];
    }
    // fluid source: 8-point Gauss rule of the point kernel along element j
    float g[4] = {0, 0, 0, 0};
    float a = (float)(0.5 * Lj), ox = (float)(mx - 0.5 * (cx + dx)), oy = (float)(my - 0.5 * (cy + dy));
    for (int q = 0; q < 8; ++q) {
        float s = (float)c_gl8x[q] * a, wt = (float)c_gl8w[q] * a;
        float zx = ox - s * tjx, zy = oy - s * tjy;
        float ir2 = 1.f / (zx * zx + zy * zy);
        pot_transient<float>(kf, zx, zy, ir2, 0.f, 0.f, 0.f, wt, wf.g_hi, 4.f * wf.ct_hi, 1.f, g);
    }
    float ss, sn;
    to_local<float>(ftx, fty, g, ss, sn);
    out[0][2] = ss; out[1][2] = sn; out[2][2] = g[3];
}

// assemble the system block of every preconditioner block:
// row (rc * m + i), column (cc * m + j), rc, cc < nc; RATE: row 1 = sigma_n + p
__global__ void k_pb_assemble(KConst<float> kf, Win<float> wf, KConst<double> kd, Win<double> wd, const double *xy,
                              int64_t N, const int32_t *boff, const int64_t *belem, const int64_t *moff, int nc, int sys,
                              float *M) {
    int b = blockIdx.y;
    int m = boff[b + 1] - boff[b];
    int64_t pair = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pair >= (int64_t)m * m) return;
    int i = (int)(pair / m), j = (int)(pair % m);
    float o[3][3];
    pair_block(kf, wf, kd, wd, xy, N, belem[boff[b] + i], belem[boff[b] + j], o);
    if (sys == DDM_SYS_RATE)
        for (int c = 0; c < 3; ++c) o[1][c] += o[2][c];
    int n = nc * m;
    float *A = M + moff[b];
    for (int rc = 0; rc < nc; ++rc)
        for (int cc = 0; cc < nc; ++cc) A[(int64_t)(rc * m + i) * n + cc * m + j] = o[rc][cc];
}

// in-place Gauss-Jordan inversion with partial pivoting, one block per matrix
__global__ void k_pb_invert(const int32_t *boff, const int64_t *moff, int nc, float *M, int *piv_ws) {
    __shared__ float sv[PT];
    __shared__ int si[PT];
    __shared__ float pivval;
    __shared__ int pivrow;
    int b = blockIdx.x;
    int n = nc * (boff[b + 1] - boff[b]);
    float *A = M + moff[b];
    int *perm = piv_ws + (int64_t)boff[b] * 3;     // column swaps to undo (n entries)
    for (int k = 0; k < n; ++k) {
        // pivot search in column k, rows >= k
        float best = -1.f;
        int bi = k;
        for (int r = k + threadIdx.x; r < n; r += PT) {
            float v = fabsf(A[(int64_t)r * n + k]);
            if (v > best) { best = v; bi = r; }
        }
        sv[threadIdx.x] = best;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int o = PT / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o && sv[threadIdx.x + o] > sv[threadIdx.x]) {
                sv[threadIdx.x] = sv[threadIdx.x + o];
                si[threadIdx.x] = si[threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            pivrow = si[0];
            perm[k] = pivrow;
        }
        __syncthreads();
        int pr = pivrow;
        if (pr != k)
            for (int c = threadIdx.x; c < n; c += PT) {
                float t = A[(int64_t)k * n + c];
                A[(int64_t)k * n + c] = A[(int64_t)pr * n + c];
                A[(int64_t)pr * n + c] = t;
            }
        __syncthreads();
        if (threadIdx.x == 0) pivval = A[(int64_t)k * n + k];
        __syncthreads();
        float ip = pivval != 0.f ? 1.f / pivval : 0.f;
        // row k: scale, with the pivot position holding the inverse pivot
        for (int c = threadIdx.x; c < n; c += PT)
            A[(int64_t)k * n + c] = (c == k) ? ip : A[(int64_t)k * n + c] * ip;
        __syncthreads();
        // eliminate column k from the other rows
        for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += PT) {
            int r = (int)(idx / n), c = (int)(idx % n);
            if (r == k || c == k) continue;
            A[idx] -= A[(int64_t)r * n + k] * A[(int64_t)k * n + c];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += PT)
            if (r != k) A[(int64_t)r * n + k] = -A[(int64_t)r * n + k] * ip;
        __syncthreads();
    }
    // undo the row interchanges as column swaps, in reverse order
    for (int k = n - 1; k >= 0; --k) {
        int pr = perm[k];
        if (pr != k)
            for (int r = threadIdx.x; r < n; r += PT) {
                float t = A[(int64_t)r * n + k];
                A[(int64_t)r * n + k] = A[(int64_t)r * n + pr];
                A[(int64_t)r * n + pr] = t;
            }
        __syncthreads();
    }
}

// z (3N layout, caller order) = Minv v (v in the system layout nc x N);
// the unknown blocks beyond nc are set to zero
__global__ void k_pb_apply(const int32_t *boff, const int64_t *belem, const int64_t *moff, int nc, const float *Minv,
                           const double *v, int64_t N, double *z, int zero_rest) {
    extern __shared__ float svf[];
    float *sv = svf;
    int b = blockIdx.x;
    int m = boff[b + 1] - boff[b], n = nc * m;
    const int64_t *el = belem + boff[b];
    for (int c = threadIdx.x; c < n; c += blockDim.x) sv[c] = (float)v[(c / m) * N + el[c % m]];
    __syncthreads();
    const float *A = Minv + moff[b];
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < n; ++c) s += A[(int64_t)r * n + c] * sv[c];
        z[(r / m) * N + el[r % m]] = (double)s;
    }
    if (zero_rest && nc < 3)
        for (int e = threadIdx.x; e < m; e += blockDim.x) z[2 * N + el[e]] = 0.0;
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
    int64_t mm = (int64_t)t->pb_max * t->pb_max;
    dim3 g((unsigned)((mm + 127) / 128), (unsigned)t->n_pblk);
    k_pb_assemble<<<g, 128, 0, s>>>(ctx->kf, wf, ctx->kd, w, t->xy_caller, t->n, t->pb_off, t->pb_elem, t->pb_moff,
                                    nc, sys, t->pb_inv);
    int *piv = nullptr;
    DDM_CUDA_TRY(ctx, dalloc(&piv, (size_t)3 * t->n * sizeof(int), s));
    k_pb_invert<<<(unsigned)t->n_pblk, PT, 0, s>>>(t->pb_off, t->pb_moff, nc, t->pb_inv, piv);
    prof_end(ctx, 8, 2);
    dfree(piv, s);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    t->pb_dt = dt;
    t->pb_sys = sys;
    return DDM_OK;
}

// z = M^-1 v : v in the system layout (nc blocks of N), z in the 3N layout
ddm_status pb_apply(ddm_ctx *ctx, ddm_tree *t, int sys, const double *v, double *z, cudaStream_t s) {
    int nc = sys == DDM_SYS_PRESSURE ? 3 : 2;
    size_t sm = (size_t)nc * t->pb_max * sizeof(float);
    k_pb_apply<<<(unsigned)t->n_pblk, 128, sm, s>>>(t->pb_off, t->pb_elem, t->pb_moff, nc, t->pb_inv, v, t->n, z, 1);
    prof_end(ctx, 8, 1);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}
