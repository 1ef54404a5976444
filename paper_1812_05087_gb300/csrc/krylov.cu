// GMRES least squares on the device, FP64 (paper Sec. 4, "modified GMRES
// with FMM products"): Givens rotations of each new Hessenberg column, the
// rotated right-hand side g, the residual estimate |g_{j+1}| with the stop
// decision of the inner cycle, and the back substitution R y = g.  One set
// of state per problem, so that the single solve (P = 1) and the lockstep
// batch share the kernels; the host reads one small status word per step.
#include <cmath>

#include "internal.h"

namespace {

// One Givens step on column j of every live problem.  hcol[p * hstride + i],
// i = 0..j+1, holds the new column (h_{0j} .. h_{j+1,j}); the rotations of
// the earlier columns are applied in order, then the new rotation zeroes
// h_{j+1,j}.  The rotated column goes into H (row-major (m + 1) x m per
// problem).  A problem leaves the cycle when |g_{j+1}| falls below its inner
// target, the column is exhausted (r = 0) or its iteration cap is reached.
__global__ void k_lsq_step(int P, int m, const double *hcol, int hstride, int j, int max_iters, double *H,
                           double *cs, double *sn, double *g, int *live, int *jend, int *iters, const double *inner,
                           double *res, int *still, double *stat, const int *err) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    if (live[p]) {
        const double *c = hcol + (int64_t)p * hstride;
        double *Hp = H + (int64_t)p * (m + 1) * m;
        const double *csp = cs + (int64_t)p * m, *snp = sn + (int64_t)p * m;
        double cur = c[0];
        for (int i = 0; i < j; ++i) {
            const double b = c[i + 1];
            Hp[(int64_t)i * m + j] = csp[i] * cur + snp[i] * b;
            cur = -snp[i] * cur + csp[i] * b;
        }
        const double b = c[j + 1];
        const double r = hypot(cur, b);
        const double cj = r > 0.0 ? cur / r : 1.0, sj = r > 0.0 ? b / r : 0.0;
        cs[(int64_t)p * m + j] = cj;
        sn[(int64_t)p * m + j] = sj;
        Hp[(int64_t)j * m + j] = r;
        double *gp = g + (int64_t)p * (m + 1);
        const double gj = gp[j];
        gp[j + 1] = -sj * gj;
        gp[j] = cj * gj;
        const int it = ++iters[p];
        jend[p] = j + 1;
        const double rj = fabs(gp[j + 1]);
        res[p] = rj;
        if (rj < inner[p] || r == 0.0 || it >= max_iters) live[p] = 0;
        else atomicAdd(still, 1);
    }
    if (stat && p == 0) {
        stat[0] = live[0];
        stat[1] = res[0];
        stat[2] = err ? (double)*err : 0.0;
    }
}

// Back substitution R y = g over the jend[p] columns of each problem, one
// warp per problem (the sum of each row across the lanes); y is zero past
// jend[p], so that a combination over more columns adds nothing.
__global__ void k_lsq_solve(int P, int m, const double *H, const double *g, const int *jend, double *y, int ystride) {
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (p >= P) return;
    const int jp = jend[p];
    const double *Hp = H + (int64_t)p * (m + 1) * m, *gp = g + (int64_t)p * (m + 1);
    double *yp = y + (int64_t)p * ystride;
    for (int k = lane; k < ystride; k += 32) yp[k] = 0.0;
    __syncwarp();
    for (int i = jp - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + lane; k < jp; k += 32) s = fma(Hp[(int64_t)i * m + k], yp[k], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) {
            const double d = Hp[(int64_t)i * m + i];
            yp[i] = d != 0.0 ? (gp[i] - s) / d : 0.0;
        }
        __syncwarp();
    }
}

// Start of a cycle: g = (beta_p, 0, ...), live = live0 && beta_p > 0,
// jend = 0, inner targets; iteration counts are kept across cycles.
__global__ void k_lsq_begin(int P, int m, const double *hbuf, double *g, int *live, int *jend, double *inner,
                            double *res) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double beta = hbuf[p], in = hbuf[P + p];
    const int l0 = hbuf[2 * P + p] != 0.0;
    double *gp = g + (int64_t)p * (m + 1);
    for (int i = 0; i <= m; ++i) gp[i] = 0.0;
    gp[0] = l0 ? beta : 0.0;
    live[p] = l0 && beta > 0.0;
    jend[p] = 0;
    inner[p] = in;
    res[p] = beta;
}

}  // namespace

void lsq_free(LsqDev &L, cudaStream_t s) {
    void *ps[] = {L.H, L.cs, L.sn, L.g, L.y, L.inner, L.res, L.stat, L.hbuf_dev, L.live, L.jend, L.iters, L.still};
    for (void *p : ps) dfree(p, s);
    if (L.hbuf) cudaFreeHost(L.hbuf);
    if (L.hstat) cudaFreeHost(L.hstat);
    if (L.hint) cudaFreeHost(L.hint);
    L = LsqDev();
}

ddm_status lsq_alloc(ddm_ctx *ctx, LsqDev &L, int P, int m, cudaStream_t s) {
    if (L.P >= P && L.m == m) return DDM_OK;
    lsq_free(L, s);
    const size_t Pz = (size_t)P;
    bool ok = dalloc(&L.H, Pz * (m + 1) * m * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.cs, Pz * m * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.sn, Pz * m * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.g, Pz * (m + 1) * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.y, Pz * (m + 2) * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.inner, Pz * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.res, Pz * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.stat, 4 * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.hbuf_dev, 3 * Pz * sizeof(double), s) == cudaSuccess &&
              dalloc(&L.live, Pz * sizeof(int), s) == cudaSuccess &&
              dalloc(&L.jend, Pz * sizeof(int), s) == cudaSuccess &&
              dalloc(&L.iters, Pz * sizeof(int), s) == cudaSuccess &&
              dalloc(&L.still, sizeof(int), s) == cudaSuccess &&
              cudaMallocHost(&L.hbuf, 3 * Pz * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&L.hstat, 2 * 4 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&L.hint, (Pz + 1) * sizeof(int)) == cudaSuccess &&
              cudaMemsetAsync(L.H, 0, Pz * (m + 1) * m * sizeof(double), s) == cudaSuccess &&
              cudaMemsetAsync(L.live, 0, Pz * sizeof(int), s) == cudaSuccess &&
              cudaMemsetAsync(L.jend, 0, Pz * sizeof(int), s) == cudaSuccess;
    if (!ok) {
        lsq_free(L, s);
        return ctx_fail(ctx, DDM_ENOMEM, "GMRES least-squares state allocation failed");
    }
    L.P = P;
    L.m = m;
    return DDM_OK;
}

ddm_status lsq_reset_iters(ddm_ctx *ctx, LsqDev &L, cudaStream_t s) {
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(L.iters, 0, (size_t)L.P * sizeof(int), s));
    return DDM_OK;
}

ddm_status lsq_begin(ddm_ctx *ctx, LsqDev &L, int P, const double *beta, const double *inner, const int *live0,
                     cudaStream_t s) {
    // the pinned staging buffer is free: every caller synchronised the
    // stream (a norm read) since the last cycle began
    for (int p = 0; p < P; ++p) {
        L.hbuf[p] = beta[p];
        L.hbuf[P + p] = inner[p];
        L.hbuf[2 * P + p] = live0 ? (double)live0[p] : 1.0;
    }
    DDM_CUDA_TRY(ctx, cudaMemcpyAsync(L.hbuf_dev, L.hbuf, 3 * (size_t)P * sizeof(double), cudaMemcpyHostToDevice, s));
    k_lsq_begin<<<(P + 127) / 128, 128, 0, s>>>(P, L.m, L.hbuf_dev, L.g, L.live, L.jend, L.inner, L.res);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

ddm_status lsq_step(ddm_ctx *ctx, LsqDev &L, int P, const double *hcol, int hstride, int j, int max_iters,
                    bool count_still, bool write_stat, cudaStream_t s) {
    if (count_still) DDM_CUDA_TRY(ctx, cudaMemsetAsync(L.still, 0, sizeof(int), s));
    k_lsq_step<<<(P + 127) / 128, 128, 0, s>>>(P, L.m, hcol, hstride, j, max_iters, L.H, L.cs, L.sn, L.g, L.live,
                                               L.jend, L.iters, L.inner, L.res, L.still,
                                               write_stat ? L.stat : nullptr, ctx->d_err);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

ddm_status lsq_solve(ddm_ctx *ctx, LsqDev &L, int P, cudaStream_t s) {
    k_lsq_solve<<<(P + 3) / 4, 128, 0, s>>>(P, L.m, L.H, L.g, L.jend, L.y, L.m + 2);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}
