// Batched products and solves of many independent (uneven) problems.
//
// A batch holds the trees of P problems.  The influence product of every
// problem is captured once into one CUDA graph (the problems' FMM kernels on
// forked streams, so that small problems overlap on the device) and the
// whole batch is advanced by one graph launch.  GMRES runs in lockstep over
// an arena that concatenates the problems' vectors: Arnoldi in FP64 with
// segmented (per-problem) reductions, then Givens rotations, convergence
// and least squares per problem on the device (krylov.cu); the host reads
// the number of problems still live after each step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "internal.h"

namespace {

constexpr int BT = 256;
constexpr int SEG_CHUNK = 2048;     // elements per reduction block
constexpr int NSTREAMS = 8;

// per reduction block: problem and element range
struct SegBlk {
    int p;
    int64_t a, b;
};

__global__ void k_dots_seg(const double *V, int64_t ld, const double *w, const SegBlk *blk, int ncols,
                           double *h /* P x ncols_stride */, int hstride) {
    __shared__ double s[BT];
    SegBlk B = blk[blockIdx.x];
    int v = blockIdx.y;
    double acc = 0.0;
    for (int64_t i = B.a + threadIdx.x; i < B.b; i += BT) acc += V[v * ld + i] * w[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = BT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&h[B.p * hstride + v], s[0]);
}
// w -= V h (per problem), hacc += h
__global__ void k_sub_seg(const double *V, int64_t ld, int nv, const double *h, int hstride, const int32_t *prob,
                          double *w, int64_t L) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= L) return;
    const double *hp = h + prob[i] * hstride;
    double s = 0.0;
    for (int v = 0; v < nv; ++v) s += hp[v] * V[v * ld + i];
    w[i] -= s;
}
__global__ void k_hacc(const double *h, double *hcol, int P, int hstride, int nv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * nv) return;
    int p = i / nv, v = i % nv;
    hcol[p * hstride + v] += h[p * hstride + v];
}
// out = w / sqrt(nrm2[p]) (0 for a zero norm); hcol[p][j1] = norm
__global__ void k_scale_seg(const double *w, const double *nrm2, const int32_t *prob, int64_t L, double *out,
                            double *hcol, int hstride, int j1, int P) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < P) hcol[i * hstride + j1] = sqrt(nrm2[i]);
    if (i >= L) return;
    double nr = sqrt(nrm2[prob[i]]);
    out[i] = nr > 0.0 ? w[i] / nr : 0.0;
}
// v0 = -w / beta[p] (0 for inactive problems: coef = 0)
__global__ void k_v0_seg(const double *w, const double *coef, const int32_t *prob, int64_t L, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= L) return;
    out[i] = coef[prob[i]] * w[i];
}
__global__ void k_axpy_b(double a, const double *x, double *y, int64_t L) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < L) y[i] += a * x[i];
}
// out_i = sum_v Y[p][v] V[v][i]
__global__ void k_comb_seg(const double *V, int64_t ld, int nv, const double *Y, int ystride, const int32_t *prob,
                           int64_t L, double *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= L) return;
    const double *yp = Y + prob[i] * ystride;
    double s = 0.0;
    for (int v = 0; v < nv; ++v) s += yp[v] * V[v * ld + i];
    out[i] = s;
}

// arena (nc blocks of N per problem) <-> 3N layout helpers, one problem
__global__ void k_copy_to3(const double *v, int64_t n, int nc, double *z3) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    for (int r = 0; r < 3; ++r) z3[r * n + e] = r < nc ? v[r * n + e] : 0.0;
}
__global__ void k_restrict_b(const double *y, int64_t n, int sys, int combine, double *out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = y[e];
    out[n + e] = y[n + e] + (combine && sys == DDM_SYS_RATE ? y[2 * n + e] : 0.0);
    if (sys == DDM_SYS_PRESSURE) out[2 * n + e] = y[2 * n + e];
}
inline unsigned nb(int64_t n) { return (unsigned)((n + BT - 1) / BT); }

// element-wise arena kernels of many problems in one launch: items
// (p, 0, a, b) cover elements [a, b) of problem p
struct SegD {
    const double *src;
    double *dst;
    int64_t n;
};
constexpr int SEG_EL = 1024;
// act (may be null): problems whose flag is 0 are skipped
__global__ void k_restrict_bb(const SegD *D, const int4 *items, int nitems, int sys, const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        if (act && !act[w.x]) continue;
        const SegD &d = D[w.x];
        for (int64_t e = w.z + threadIdx.x; e < w.w; e += BT) {
            d.dst[e] = d.src[e];
            d.dst[d.n + e] = d.src[d.n + e] + (sys == DDM_SYS_RATE ? d.src[2 * d.n + e] : 0.0);
            if (sys == DDM_SYS_PRESSURE) d.dst[2 * d.n + e] = d.src[2 * d.n + e];
        }
    }
}
__global__ void k_copy3_bb(const SegD *D, const int4 *items, int nitems, int nc, const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        if (act && !act[w.x]) continue;
        const SegD &d = D[w.x];
        for (int64_t e = w.z + threadIdx.x; e < w.w; e += BT)
            for (int r = 0; r < 3; ++r) d.dst[r * d.n + e] = r < nc ? d.src[r * d.n + e] : 0.0;
    }
}
// dst += src on the first nc blocks of each problem's 3N layout
__global__ void k_axpy3_bb(const SegD *D, const int4 *items, int nitems, int nc, const int *act) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        if (act && !act[w.x]) continue;
        const SegD &d = D[w.x];
        for (int64_t e = w.z + threadIdx.x; e < w.w; e += BT)
            for (int r = 0; r < nc; ++r) d.dst[r * d.n + e] += d.src[r * d.n + e];
    }
}

}  // namespace

// arena segments of many problems (device descriptors and element items)
struct SegBatch {
    SegD *desc = nullptr;
    int4 *items = nullptr;
    int n = 0;
    void release(cudaStream_t s) {
        dfree(desc, s);
        dfree(items, s);
        desc = nullptr;
        items = nullptr;
        n = 0;
    }
};

struct ddm_batch {
    int P = 0;
    std::vector<ddm_tree *> trees;
    std::vector<int64_t> N, off3;         // elements, offset of each problem in 3N-layout arenas
    int64_t tot3 = 0;
    // solver arena (system rows)
    int nc = 3, sys = -1, m = 0;
    std::vector<int64_t> offs;            // offset of each problem in the system arena
    int64_t L = 0;
    int32_t *prob = nullptr;              // arena index -> problem
    SegBlk *blk = nullptr;
    int nblk = 0;
    double *V = nullptr, *w = nullptr, *vin = nullptr, *b = nullptr, *tmp = nullptr;
    double *full = nullptr, *y3 = nullptr, *Minv = nullptr;
    double *h = nullptr, *hcol = nullptr, *nrm = nullptr, *coef = nullptr;
    LsqDev lsq;                           // device least squares of every problem
    std::vector<int64_t> minv_off;
    // graphs
    cudaGraphExec_t g_op = nullptr, g_prod = nullptr, g_res = nullptr;
    double g_op_dt = -1, g_prod_dt = -1, g_res_dt = -1;
    int g_op_mode = -1, g_prod_mode = -1, g_res_mode = -1, g_op_sys = -1, g_res_sys = -1;
    const double *g_prod_x = nullptr, *g_res_x = nullptr;
    long long k_op = 0, k_prod = 0, k_res = 0;   // kernels per graph launch
    std::vector<int> op_set;                     // problems in g_op / g_res
    double *g_prod_y = nullptr;
    cudaStream_t fork[NSTREAMS] = {};
    cudaStream_t cap = nullptr;
    cudaStream_t ast = nullptr;            // stream of the arena allocations
    cudaEvent_t ev_fork[NSTREAMS] = {}, ev_join[NSTREAMS] = {};
    // work lists of the one-launch-per-stage graphs (product, Arnoldi
    // operator, residual): FMM products grouped by order, preconditioner,
    // arena copies and restrictions
    std::vector<BatchFmm *> bf[3];          // 0 product, 1 Arnoldi operator, 2 residual
    BatchPb *bp = nullptr, *bpx = nullptr;  // preconditioner of the Arnoldi operator / of the update of x
    SegBatch seg[5];                        // 1 operator restriction, 2 residual copy, 3 residual
                                            // restriction, 4 update of x
    int *d_act = nullptr, *h_act = nullptr; // 3P flags (device, pinned host): FMM products of the
                                            // operator, FMM products of the residual, problems still active
    void free_lists(int k) {
        for (BatchFmm *f : bf[k]) bfmm_free(f, ast);
        bf[k].clear();
        if (k == 1) {
            seg[1].release(ast);
            seg[4].release(ast);
            if (bp) { bpb_free(bp, ast); bp = nullptr; }
            if (bpx) { bpb_free(bpx, ast); bpx = nullptr; }
        }
        if (k == 2) { seg[2].release(ast); seg[3].release(ast); }
    }
    void free_solver() {
        void *ps[] = {prob, blk, V, w, vin, b, tmp, Minv, h, hcol, nrm, coef, d_act};
        for (void *p : ps) dfree(p, ast);
        if (h_act) cudaFreeHost(h_act);
        h_act = nullptr;
        d_act = nullptr;
        lsq_free(lsq, ast);
        prob = nullptr; blk = nullptr; V = w = vin = b = tmp = Minv = h = hcol = nrm = coef = nullptr;
        sys = -1; m = 0;
    }
    void free_graphs() {
        if (g_op) cudaGraphExecDestroy(g_op);
        if (g_prod) cudaGraphExecDestroy(g_prod);
        if (g_res) cudaGraphExecDestroy(g_res);
        g_op = g_prod = g_res = nullptr;
        for (int k = 0; k < 3; ++k) free_lists(k);
    }
};

namespace {

// capture fn(p, stream) for every problem into one graph on ctx->stream
template <class Fn>
ddm_status capture(ddm_ctx *ctx, ddm_batch *B, cudaGraphExec_t *out, long long *kernels, const std::vector<int> &idx,
                   Fn fn) {
    // capture on the batch's own stream; the graph is launched on the context stream
    cudaStream_t s = B->cap;
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (*out) { cudaGraphExecDestroy(*out); *out = nullptr; }
    cudaGraph_t g;
    long long before[DDM_NSTAGES];
    for (int k = 0; k < DDM_NSTAGES; ++k) before[k] = ctx->prof.launches[k];
    DDM_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaEvent_t e0;
    cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
    cudaEventRecord(e0, s);
    int ns = std::max(1, std::min<int>(NSTREAMS, (int)idx.size()));
    for (int k = 0; k < ns; ++k) cudaStreamWaitEvent(B->fork[k], e0, 0);
    ddm_status st = DDM_OK;
    for (size_t q = 0; q < idx.size() && st == DDM_OK; ++q) st = fn(idx[q], B->fork[q % ns]);
    for (int k = 0; k < ns; ++k) {
        cudaEventRecord(B->ev_join[k], B->fork[k]);
        cudaStreamWaitEvent(s, B->ev_join[k], 0);
    }
    cudaError_t e = cudaStreamEndCapture(s, &g);
    cudaEventDestroy(e0);
    long long kern = 0;
    for (int k = 0; k < DDM_NSTAGES; ++k) { kern += ctx->prof.launches[k] - before[k]; ctx->prof.launches[k] = before[k]; }
    *kernels = kern;
    if (st) { if (e == cudaSuccess) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return ctx_fail(ctx, DDM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ctx_fail(ctx, DDM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return DDM_OK;
}

// run every problem's product once outside capture so that per-tree caches
// (workspaces, M2L operators, own-element blocks) exist before capture
ddm_status warm(ddm_ctx *ctx, ddm_batch *B, double dt, int mode) {
    for (int p = 0; p < B->P; ++p) {
        ddm_status st = op_apply(ctx, B->trees[p], 0.0, dt, B->full + B->off3[p], B->y3 + B->off3[p], mode, 0, 1.0);
        if (st) return st;
    }
    return DDM_OK;
}

ddm_status seg_build(ddm_ctx *ctx, ddm_batch *B, const std::vector<int> &idx, const double *src, const int64_t *soff,
                     double *dst, const int64_t *doff, SegBatch &out) {
    std::vector<SegD> hd(B->P);
    std::vector<int4> hi;
    for (int p = 0; p < B->P; ++p) hd[p] = SegD{src + soff[p], dst + doff[p], B->N[p]};
    for (int p : idx)
        for (int64_t a = 0; a < B->N[p]; a += SEG_EL)
            hi.push_back(make_int4(p, 0, (int)a, (int)std::min<int64_t>(B->N[p], a + SEG_EL)));
    out.release(B->ast);
    cudaStream_t s = B->ast;
    bool ok = dalloc(&out.desc, hd.size() * sizeof(SegD), s) == cudaSuccess &&
              dalloc(&out.items, std::max<size_t>(1, hi.size()) * sizeof(int4), s) == cudaSuccess &&
              cudaMemcpyAsync(out.desc, hd.data(), hd.size() * sizeof(SegD), cudaMemcpyHostToDevice, s) == cudaSuccess &&
              (hi.empty() || cudaMemcpyAsync(out.items, hi.data(), hi.size() * sizeof(int4), cudaMemcpyHostToDevice, s) ==
                                 cudaSuccess) &&
              cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) return ctx_fail(ctx, DDM_ENOMEM, "batch: arena work list allocation failed");
    out.n = (int)hi.size();
    return DDM_OK;
}

// products y_p = [K(dt)] x_p of the problems in idx whose mode is plain FMM,
// grouped by Chebyshev order: one work-list set per order
ddm_status fmm_groups(ddm_ctx *ctx, ddm_batch *B, const std::vector<int> &idx, double dt, const double *x,
                      const int64_t *xoff, double *y, std::vector<BatchFmm *> &out, const int *act = nullptr) {
    std::map<int, std::vector<int>> by_n;
    for (int p : idx) by_n[B->trees[p]->prm.n_cheb].push_back(p);
    std::vector<const double *> xs(B->P);
    std::vector<double *> ys(B->P);
    for (int p = 0; p < B->P; ++p) {
        xs[p] = x + xoff[p];
        ys[p] = y + B->off3[p];
    }
    for (auto &g : by_n) {
        BatchFmm *f = nullptr;
        ddm_status st = bfmm_build(ctx, B->trees.data(), B->P, g.second.data(), (int)g.second.size(), 0.0, dt,
                                   xs.data(), ys.data(), act, B->ast, &f);
        if (st) return st;
        out.push_back(f);
    }
    return DDM_OK;
}

// capture body() on the batch's capture stream into one graph (the FMM far
// branch may fork to B->fork[0])
template <class Fn>
ddm_status capture_seq(ddm_ctx *ctx, ddm_batch *B, cudaGraphExec_t *out, long long *kernels, Fn body) {
    cudaStream_t s = B->cap;
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (*out) { cudaGraphExecDestroy(*out); *out = nullptr; }
    long long before[DDM_NSTAGES];
    for (int k = 0; k < DDM_NSTAGES; ++k) before[k] = ctx->prof.launches[k];
    cudaGraph_t g;
    DDM_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    ddm_status st = body(s);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    long long kern = 0;
    for (int k = 0; k < DDM_NSTAGES; ++k) { kern += ctx->prof.launches[k] - before[k]; ctx->prof.launches[k] = before[k]; }
    *kernels = kern;
    if (st) { if (e == cudaSuccess) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return ctx_fail(ctx, DDM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ctx_fail(ctx, DDM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return DDM_OK;
}

inline unsigned seg_grid(int n) { return (unsigned)std::max(1, std::min(n, 152 * 8)); }

// per-problem products (escalated precision) inside a capture, spread over
// the batch's forked streams 1.. so that they overlap each other and the
// batched stages on the capture stream and fork stream 0
template <class Fn>
ddm_status fork_each(ddm_ctx *ctx, ddm_batch *B, cudaStream_t cs, const std::vector<int> &idx, Fn fn) {
    if (idx.empty()) return DDM_OK;
    const int ns = std::max(1, std::min<int>(NSTREAMS - 1, (int)idx.size()));
    DDM_CUDA_TRY(ctx, cudaEventRecord(B->ev_fork[0], cs));
    for (int k = 0; k < ns; ++k) DDM_CUDA_TRY(ctx, cudaStreamWaitEvent(B->fork[1 + k], B->ev_fork[0], 0));
    for (size_t q = 0; q < idx.size(); ++q) {
        ddm_status e = fn(idx[q], B->fork[1 + q % ns]);
        if (e) return e;
    }
    for (int k = 0; k < ns; ++k) {
        DDM_CUDA_TRY(ctx, cudaEventRecord(B->ev_join[1 + k], B->fork[1 + k]));
        DDM_CUDA_TRY(ctx, cudaStreamWaitEvent(cs, B->ev_join[1 + k], 0));
    }
    return DDM_OK;
}

}  // namespace

extern "C" {

ddm_status ddm_batch_create(ddm_ctx *ctx, ddm_tree *const *trees, int n, ddm_batch **out) {
    if (!ctx || !trees || n <= 0 || !out) return ctx_fail(ctx, DDM_EINVAL, "ddm_batch_create: bad arguments");
    ddm_batch *B = new ddm_batch();
    B->P = n;
    int64_t o = 0;
    for (int p = 0; p < n; ++p) {
        if (!trees[p]) { delete B; return ctx_fail(ctx, DDM_EINVAL, "ddm_batch_create: null tree"); }
        B->trees.push_back(trees[p]);
        B->N.push_back(trees[p]->n);
        B->off3.push_back(o);
        o += 3 * trees[p]->n;
    }
    B->tot3 = o;
    B->ast = ctx->stream;
    if (dalloc(&B->full, o * sizeof(double), B->ast) != cudaSuccess || dalloc(&B->y3, o * sizeof(double), B->ast) != cudaSuccess) {
        delete B;
        return ctx_fail(ctx, DDM_ENOMEM, "batch arena allocation failed");
    }
    cudaMemsetAsync(B->full, 0, o * sizeof(double), B->ast);
    cudaMemsetAsync(B->y3, 0, o * sizeof(double), B->ast);
    cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    for (int k = 0; k < NSTREAMS; ++k) {
        cudaStreamCreateWithFlags(&B->fork[k], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&B->ev_join[k], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&B->ev_fork[k], cudaEventDisableTiming);
    }
    *out = B;
    return DDM_OK;
}

void ddm_batch_destroy(ddm_batch *B) {
    if (!B) return;
    B->free_graphs();
    B->free_solver();
    dfree(B->full, B->ast);
    dfree(B->y3, B->ast);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (int k = 0; k < NSTREAMS; ++k) {
        if (B->fork[k]) cudaStreamDestroy(B->fork[k]);
        if (B->ev_join[k]) cudaEventDestroy(B->ev_join[k]);
        if (B->ev_fork[k]) cudaEventDestroy(B->ev_fork[k]);
    }
    delete B;
}

ddm_status ddm_batch_matvec(ddm_ctx *ctx, ddm_batch *B, double dt, const double *d_x, double *d_y, int mode) {
    if (!ctx || !B || !d_x || !d_y || !(dt > 0)) return ctx_fail(ctx, DDM_EINVAL, "ddm_batch_matvec: bad arguments");
    ddm_status st = upload_tables(ctx);
    if (st) return st;
    if (!B->g_prod || B->g_prod_dt != dt || B->g_prod_mode != mode || B->g_prod_x != d_x || B->g_prod_y != d_y) {
        int saved = ctx->prof.on;
        ctx->prof.on = 0;
        std::vector<int> all(B->P);
        for (int p = 0; p < B->P; ++p) all[p] = p;
        if (mode == DDM_MODE_FMM) {
            // one launch per stage over every problem (work lists by order)
            B->free_lists(0);
            st = fmm_groups(ctx, B, all, dt, d_x, B->off3.data(), d_y, B->bf[0]);
            if (!st)
                st = capture_seq(ctx, B, &B->g_prod, &B->k_prod, [&](cudaStream_t cs) -> ddm_status {
                    for (BatchFmm *f : B->bf[0]) {
                        ddm_status e = bfmm_launch(ctx, f, cs, B->fork[0]);
                        if (e) return e;
                    }
                    return DDM_OK;
                });
        } else {
            if ((st = warm(ctx, B, dt, mode))) { ctx->prof.on = saved; return st; }
            DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            st = capture(ctx, B, &B->g_prod, &B->k_prod, all, [&](int p, cudaStream_t s) {
                return op_apply(ctx, B->trees[p], 0.0, dt, d_x + B->off3[p], d_y + B->off3[p], mode, 0, 1.0, s);
            });
        }
        ctx->prof.on = saved;
        if (st) return st;
        B->g_prod_dt = dt; B->g_prod_mode = mode; B->g_prod_x = d_x; B->g_prod_y = d_y;
    }
    DDM_CUDA_TRY(ctx, cudaGraphLaunch(B->g_prod, ctx->stream));
    prof_end(ctx, 6, (int)B->k_prod);
    return DDM_OK;
}

ddm_status ddm_batch_gmres_solve(ddm_ctx *ctx, ddm_batch *B, double dt, const double *d_rhs, double *d_x,
                                 const ddm_gmres_params *prm, ddm_gmres_info *infos) {
    if (!ctx || !B || !d_rhs || !d_x || !(dt > 0)) return ctx_fail(ctx, DDM_EINVAL, "ddm_batch_gmres_solve: bad arguments");
    ddm_gmres_params Pm = prm ? *prm : ddm_gmres_params{DDM_SYS_PRESSURE, 50, 1000, 1e-6, DDM_MODE_FMM};
    if (Pm.restart <= 0) Pm.restart = 50;
    if (Pm.max_iters <= 0) Pm.max_iters = 1000;
    if (!(Pm.tol > 0)) Pm.tol = 1e-6;
    if (Pm.system < 0 || Pm.system > 2 || Pm.restart > 500) return ctx_fail(ctx, DDM_EINVAL, "bad GMRES params");
    ddm_status st = upload_tables(ctx);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    const int P = B->P, m = Pm.restart, sys = Pm.system, mode = Pm.mode & ~DDM_MODE_PRECISE;
    const int nc = sys == DDM_SYS_PRESSURE ? 3 : 2;
    const int hs = m + 2;
    // (re)allocate the solver arena
    if (B->sys != sys || B->m < m) {
        B->free_solver();
        B->free_graphs();
        B->nc = nc;
        B->offs.assign(P + 1, 0);
        B->minv_off.assign(P + 1, 0);
        for (int p = 0; p < P; ++p) {
            B->offs[p + 1] = B->offs[p] + nc * B->N[p];
            B->minv_off[p + 1] = B->minv_off[p] + 9 * B->N[p];
        }
        int64_t L = B->offs[P];
        B->L = L;
        std::vector<int32_t> hp(L);
        std::vector<SegBlk> hb;
        for (int p = 0; p < P; ++p) {
            for (int64_t i = B->offs[p]; i < B->offs[p + 1]; ++i) hp[i] = p;
            for (int64_t a = B->offs[p]; a < B->offs[p + 1]; a += SEG_CHUNK)
                hb.push_back(SegBlk{p, a, std::min(a + SEG_CHUNK, B->offs[p + 1])});
        }
        B->nblk = (int)hb.size();
        bool ok = dalloc(&B->prob, L * sizeof(int32_t), s) == cudaSuccess &&
                  dalloc(&B->blk, hb.size() * sizeof(SegBlk), s) == cudaSuccess &&
                  dalloc(&B->V, (size_t)(m + 1) * L * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->w, L * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->vin, L * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->b, L * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->tmp, L * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->Minv, B->minv_off[P] * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->h, (size_t)P * hs * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->hcol, (size_t)P * hs * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->nrm, (size_t)P * hs * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->coef, P * sizeof(double), s) == cudaSuccess &&
                  dalloc(&B->d_act, 3 * (size_t)P * sizeof(int), s) == cudaSuccess &&
                  cudaMallocHost(&B->h_act, 3 * (size_t)P * sizeof(int)) == cudaSuccess;
        if (!ok) { B->free_solver(); return ctx_fail(ctx, DDM_ENOMEM, "batch GMRES arena allocation failed"); }
        cudaMemcpyAsync(B->prob, hp.data(), L * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(B->blk, hb.data(), hb.size() * sizeof(SegBlk), cudaMemcpyHostToDevice, s);
        B->sys = sys;
        B->m = m;
        DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    const int64_t L = B->L;
    // preconditioner blocks per problem (inverted fracture-chain blocks)
    for (int p = 0; p < P; ++p)
        if ((st = pb_prepare(ctx, B->trees[p], dt, sys, s, true))) return st;
    if ((st = pc_invert_many(ctx, B->trees.data(), P, s))) return st;
    // graphs: preconditioned operator vin -> w, residual operator (precise) x -> tmp
    int saved = ctx->prof.on;
    ctx->prof.on = 0;
    // per problem precision level, as in ddm_gmres_solve: 0 requested
    // products throughout, 1 precise residuals, 2 precise inner products too
    std::vector<int> level(P, 0);
    // Plain-FMM solves: every stage of all problems' operator (preconditioner,
    // product, restriction) and of their residual is one launch over a work
    // list built once per solve and captured once; per-problem flags on the
    // device select the problems each launch computes (still active, plain
    // or escalated precision), so nothing is rebuilt as problems converge.
    // Problems whose precision escalated take their own products, launched
    // beside the graphs on the batch's forked streams.
    const bool batched = mode == DDM_MODE_FMM;
    int *act_op = B->d_act, *act_res = B->d_act + P, *act_all = B->d_act + 2 * P;
    auto build_batched = [&]() -> ddm_status {
        B->free_lists(1);
        B->free_lists(2);
        std::vector<int> all(P);
        std::vector<const double *> vs(P), ts(P);
        std::vector<double *> zs(P);
        for (int p = 0; p < P; ++p) {
            all[p] = p;
            vs[p] = B->vin + B->offs[p];
            ts[p] = B->tmp + B->offs[p];
            zs[p] = B->full + B->off3[p];
        }
        ddm_status e = bpb_build(ctx, B->trees.data(), P, sys, vs.data(), zs.data(), act_all, B->ast, &B->bp);
        if (!e) e = bpb_build(ctx, B->trees.data(), P, sys, ts.data(), zs.data(), act_all, B->ast, &B->bpx);
        if (!e) e = fmm_groups(ctx, B, all, dt, B->full, B->off3.data(), B->y3, B->bf[1], act_op);
        if (!e) e = fmm_groups(ctx, B, all, dt, B->full, B->off3.data(), B->y3, B->bf[2], act_res);
        if (!e) e = seg_build(ctx, B, all, B->y3, B->off3.data(), B->w, B->offs.data(), B->seg[1]);
        if (!e) e = seg_build(ctx, B, all, d_x, B->off3.data(), B->full, B->off3.data(), B->seg[2]);
        if (!e) e = seg_build(ctx, B, all, B->y3, B->off3.data(), B->tmp, B->offs.data(), B->seg[3]);
        if (!e) e = seg_build(ctx, B, all, B->full, B->off3.data(), d_x, B->off3.data(), B->seg[4]);
        if (e) return e;
        e = capture_seq(ctx, B, &B->g_op, &B->k_op, [&](cudaStream_t cs) -> ddm_status {
            ddm_status r = bpb_launch(ctx, B->bp, cs);
            for (BatchFmm *f : B->bf[1])
                if (!r) r = bfmm_launch(ctx, f, cs, B->fork[0]);
            return r;
        });
        if (e) return e;
        return capture_seq(ctx, B, &B->g_res, &B->k_res, [&](cudaStream_t cs) -> ddm_status {
            k_copy3_bb<<<seg_grid(B->seg[2].n), BT, 0, cs>>>(B->seg[2].desc, B->seg[2].items, B->seg[2].n, nc,
                                                            act_all);
            prof_end(ctx, 8, 1);
            ddm_status r = DDM_OK;
            for (BatchFmm *f : B->bf[2])
                if (!r) r = bfmm_launch(ctx, f, cs, B->fork[0]);
            return r;
        });
    };
    auto capture_op = [&](const std::vector<int> &idx) -> ddm_status {
        return capture(ctx, B, &B->g_op, &B->k_op, idx, [&](int p, cudaStream_t ps) -> ddm_status {
            int64_t n = B->N[p];
            ddm_status e = pb_apply(ctx, B->trees[p], sys, B->vin + B->offs[p], B->full + B->off3[p], ps);
            if (e) return e;
            e = op_apply(ctx, B->trees[p], 0.0, dt, B->full + B->off3[p], B->y3 + B->off3[p],
                         arnoldi_mode(mode, level[p], n), 0, 1.0, ps);
            if (e) return e;
            k_restrict_b<<<nb(n), BT, 0, ps>>>(B->y3 + B->off3[p], n, sys, 1, B->w + B->offs[p]);
            return DDM_OK;
        });
    };
    auto capture_res = [&](const std::vector<int> &idx) -> ddm_status {
        return capture(ctx, B, &B->g_res, &B->k_res, idx, [&](int p, cudaStream_t ps) -> ddm_status {
            int64_t n = B->N[p];
            k_copy_to3<<<nb(n), BT, 0, ps>>>(d_x + B->off3[p], n, nc, B->full + B->off3[p]);
            ddm_status e = op_apply(ctx, B->trees[p], 0.0, dt, B->full + B->off3[p], B->y3 + B->off3[p],
                                    residual_mode(mode, level[p], n), 0, 1.0, ps);
            if (e) return e;
            k_restrict_b<<<nb(n), BT, 0, ps>>>(B->y3 + B->off3[p], n, sys, 1, B->tmp + B->offs[p]);
            return DDM_OK;
        });
    };
    std::vector<int> every(P);
    for (int p = 0; p < P; ++p) every[p] = p;
    if (!batched && ((st = warm(ctx, B, dt, mode)) || (st = warm(ctx, B, dt, mode | DDM_MODE_PRECISE)))) {
        ctx->prof.on = saved;
        return st;
    }
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (batched) st = build_batched();
    else if (!(st = capture_op(every))) st = capture_res(every);
    if (st) { ctx->prof.on = saved; return st; }
    B->op_set = every;
    ctx->prof.on = saved;
    // b = restrict(rhs) (- restrict(A [0; 0; Dq]) for the 2N systems)
    for (int p = 0; p < P; ++p) {
        int64_t n = B->N[p];
        k_restrict_b<<<nb(n), BT, 0, s>>>(d_rhs + B->off3[p], n, sys, 1, B->b + B->offs[p]);
        if (sys != DDM_SYS_PRESSURE) {
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(B->full + B->off3[p], 0, 2 * n * sizeof(double), s));
            DDM_CUDA_TRY(ctx, cudaMemcpyAsync(B->full + B->off3[p] + 2 * n, d_x + B->off3[p] + 2 * n, n * sizeof(double),
                                              cudaMemcpyDeviceToDevice, s));
            if ((st = op_apply(ctx, B->trees[p], 0.0, dt, B->full + B->off3[p], B->y3 + B->off3[p],
                               mode | DDM_MODE_PRECISE, 0, 1.0)))
                return st;
            k_restrict_b<<<nb(n), BT, 0, s>>>(B->y3 + B->off3[p], n, sys, 1, B->tmp + B->offs[p]);
            k_axpy_b<<<nb(nc * n), BT, 0, s>>>(-1.0, B->tmp + B->offs[p], B->b + B->offs[p], nc * n);
        }
    }
    auto seg_norms = [&](const double *v, std::vector<double> &out) -> ddm_status {
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(B->nrm, 0, P * sizeof(double), s));
        k_dots_seg<<<dim3(B->nblk, 1), BT, 0, s>>>(v, 0, v, B->blk, 1, B->nrm, 1);
        out.resize(P);
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(out.data(), B->nrm, P * sizeof(double), cudaMemcpyDeviceToHost, s));
        DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        for (double &x : out) x = sqrt(x);
        return DDM_OK;
    };
    std::vector<double> bn, beta;
    if ((st = seg_norms(B->b, bn))) return st;
    for (double &x : bn)
        if (x == 0) x = 1;
    std::vector<int> iters(P, 0), restarts(P, 0), conv(P, 0), stall(P, 0), active(P, 1);
    std::vector<double> rel(P, 1e300), best(P, 1e300), coef(P), inner(P);
    if ((st = lsq_alloc(ctx, B->lsq, P, m, s)) || (st = lsq_reset_iters(ctx, B->lsq, s))) return st;
    int *h_still = B->lsq.hint, *h_iters = B->lsq.hint + 1;
    int total = 0;
    // batched: the flags of the launches (the pinned mirror is only rewritten
    // after a synchronisation, when its previous copy is complete)
    auto set_flags = [&]() -> ddm_status {
        for (int p = 0; p < P; ++p) {
            B->h_act[p] = active[p] && level[p] < 2;
            B->h_act[P + p] = active[p] && residual_mode(mode, level[p], B->N[p]) == DDM_MODE_FMM;
            B->h_act[2 * P + p] = active[p];
        }
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(B->d_act, B->h_act, 3 * (size_t)P * sizeof(int), cudaMemcpyHostToDevice, s));
        return DDM_OK;
    };
    std::vector<int> prec_op, other_res;
    auto escalated = [&]() {
        prec_op.clear();
        other_res.clear();
        for (int p = 0; p < P; ++p) {
            if (!active[p]) continue;
            if (level[p] >= 2) prec_op.push_back(p);
            if (residual_mode(mode, level[p], B->N[p]) != DDM_MODE_FMM) other_res.push_back(p);
        }
    };
    while (true) {
        // residuals (operator of each problem's level): tmp = A x, w = A x - b
        if (batched) {
            escalated();
            if ((st = set_flags())) return st;
            DDM_CUDA_TRY(ctx, cudaGraphLaunch(B->g_res, s));
            st = fork_each(ctx, B, s, other_res, [&](int p, cudaStream_t ps) {
                return op_apply(ctx, B->trees[p], 0.0, dt, B->full + B->off3[p], B->y3 + B->off3[p],
                                residual_mode(mode, level[p], B->N[p]), 0, 1.0, ps);
            });
            if (st) return st;
            k_restrict_bb<<<seg_grid(B->seg[3].n), BT, 0, s>>>(B->seg[3].desc, B->seg[3].items, B->seg[3].n, sys,
                                                             act_all);
        } else {
            DDM_CUDA_TRY(ctx, cudaGraphLaunch(B->g_res, s));
        }
        prof_end(ctx, 6, (int)B->k_res);
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(B->w, B->tmp, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
        k_axpy_b<<<nb(L), BT, 0, s>>>(-1.0, B->b, B->w, L);
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(h_iters, B->lsq.iters, P * sizeof(int), cudaMemcpyDeviceToHost, s));
        if ((st = seg_norms(B->w, beta))) return st;      // synchronises: h_iters is current
        std::copy(h_iters, h_iters + P, iters.begin());
        int nact = 0;
        bool reprec = false;
        std::vector<int> remeasure(P, 0);   // switched to precise residuals: no cycle until re-measured
        for (int p = 0; p < P; ++p) {
            if (!active[p]) continue;
            rel[p] = beta[p] / bn[p];
            if (rel[p] < Pm.tol) { conv[p] = 1; active[p] = 0; continue; }
            if (rel[p] < 0.9 * best[p]) { best[p] = rel[p]; stall[p] = 0; }
            else if (level[p] < max_level(B->N[p])) {
                if (++level[p] == 1) { best[p] = 1e300; remeasure[p] = 1; }
                stall[p] = 0;
                reprec = true;
            }
            else if (++stall[p] >= 3) { active[p] = 0; continue; }
            if (iters[p] >= Pm.max_iters) { active[p] = 0; continue; }
            ++nact;
        }
        if (nact == 0 || total >= Pm.max_iters) break;
        // drop converged problems from the graphs once a quarter of them left
        // (and re-capture when a problem switched to precise inner products)
        if (batched) {
            escalated();
            if ((st = set_flags())) return st;
        } else if (reprec || nact < 0.75 * (double)B->op_set.size()) {
            std::vector<int> act;
            for (int p = 0; p < P; ++p)
                if (active[p]) act.push_back(p);
            int sv2 = ctx->prof.on;
            ctx->prof.on = 0;
            if ((st = capture_op(act)) || (st = capture_res(act))) { ctx->prof.on = sv2; return st; }
            ctx->prof.on = sv2;
            B->op_set = act;
        }
        for (int p = 0; p < P; ++p) coef[p] = active[p] && beta[p] > 0 ? -1.0 / beta[p] : 0.0;
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(B->coef, coef.data(), P * sizeof(double), cudaMemcpyHostToDevice, s));
        k_v0_seg<<<nb(L), BT, 0, s>>>(B->w, B->coef, B->prob, L, B->V);
        std::vector<int> live(P);
        for (int p = 0; p < P; ++p) {
            live[p] = active[p] && !remeasure[p];
            inner[p] = level[p] == 0 ? 0.3 * Pm.tol * bn[p] : std::max(0.3 * Pm.tol * bn[p], 1e-4 * beta[p]);
        }
        if ((st = lsq_begin(ctx, B->lsq, P, beta.data(), inner.data(), live.data(), s))) return st;
        int j = 0;
        for (; j < m; ++j) {
            DDM_CUDA_TRY(ctx, cudaMemcpyAsync(B->vin, B->V + (int64_t)j * L, L * sizeof(double), cudaMemcpyDeviceToDevice, s));
            DDM_CUDA_TRY(ctx, cudaGraphLaunch(B->g_op, s));
            if (batched) {
                st = fork_each(ctx, B, s, prec_op, [&](int p, cudaStream_t ps) {
                    return op_apply(ctx, B->trees[p], 0.0, dt, B->full + B->off3[p], B->y3 + B->off3[p],
                                    arnoldi_mode(mode, level[p], B->N[p]), 0, 1.0, ps);
                });
                if (st) return st;
                k_restrict_bb<<<seg_grid(B->seg[1].n), BT, 0, s>>>(B->seg[1].desc, B->seg[1].items, B->seg[1].n,
                                                                 sys, act_all);
            }
            prof_end(ctx, 6, (int)B->k_op);
            prof_end(ctx, 8, 10);
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(B->hcol, 0, (size_t)P * hs * sizeof(double), s));
            for (int pass = 0; pass < 2; ++pass) {
                DDM_CUDA_TRY(ctx, cudaMemsetAsync(B->h, 0, (size_t)P * hs * sizeof(double), s));
                k_dots_seg<<<dim3(B->nblk, j + 1), BT, 0, s>>>(B->V, L, B->w, B->blk, j + 1, B->h, hs);
                k_sub_seg<<<nb(L), BT, 0, s>>>(B->V, L, j + 1, B->h, hs, B->prob, B->w, L);
                k_hacc<<<nb((int64_t)P * (j + 1)), BT, 0, s>>>(B->h, B->hcol, P, hs, j + 1);
            }
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(B->nrm, 0, P * sizeof(double), s));
            k_dots_seg<<<dim3(B->nblk, 1), BT, 0, s>>>(B->w, 0, B->w, B->blk, 1, B->nrm, 1);
            k_scale_seg<<<nb(std::max<int64_t>(L, P)), BT, 0, s>>>(B->w, B->nrm, B->prob, L, B->V + (int64_t)(j + 1) * L,
                                                                   B->hcol, hs, j + 1, P);
            // Givens step of every live problem on the device; read how many stay live
            if ((st = lsq_step(ctx, B->lsq, P, B->hcol, hs, j, Pm.max_iters, true, false, s))) return st;
            DDM_CUDA_TRY(ctx, cudaMemcpyAsync(h_still, B->lsq.still, sizeof(int), cudaMemcpyDeviceToHost, s));
            DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            ++total;
            if (*h_still == 0) { ++j; break; }
        }
        // per-problem least squares on the device and update x += M^-1 V y
        if ((st = lsq_solve(ctx, B->lsq, P, s))) return st;
        for (int p = 0; p < P; ++p)
            if (active[p]) ++restarts[p];
        if (j > 0 && batched) {
            k_comb_seg<<<nb(L), BT, 0, s>>>(B->V, L, j, B->lsq.y, m + 2, B->prob, L, B->tmp);
            if ((st = bpb_launch(ctx, B->bpx, s))) return st;
            k_axpy3_bb<<<seg_grid(B->seg[4].n), BT, 0, s>>>(B->seg[4].desc, B->seg[4].items, B->seg[4].n, nc,
                                                          act_all);
        } else if (j > 0) {
            k_comb_seg<<<nb(L), BT, 0, s>>>(B->V, L, j, B->lsq.y, m + 2, B->prob, L, B->tmp);
            for (int p = 0; p < P; ++p)
                if (active[p]) {
                    if ((st = pb_apply(ctx, B->trees[p], sys, B->tmp + B->offs[p], B->full + B->off3[p], s))) return st;
                    k_axpy_b<<<nb(nc * B->N[p]), BT, 0, s>>>(1.0, B->full + B->off3[p], d_x + B->off3[p], nc * B->N[p]);
                }
        }
    }
    DDM_CUDA_TRY(ctx, cudaMemcpyAsync(h_iters, B->lsq.iters, P * sizeof(int), cudaMemcpyDeviceToHost, s));
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    std::copy(h_iters, h_iters + P, iters.begin());
    bool all = true;
    for (int p = 0; p < P; ++p) {
        if (infos) {
            infos[p].iterations = iters[p];
            infos[p].restarts = restarts[p];
            infos[p].rel_residual = rel[p];
            infos[p].converged = conv[p];
        }
        all = all && conv[p];
    }
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return all ? DDM_OK : ctx_fail(ctx, DDM_ENOTCONV, "batched GMRES: some problems did not converge");
}

}  // extern "C"
