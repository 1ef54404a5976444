// Autotuner of the FMM parameters (no counterpart in the paper).
//
// For one representative problem (a size bucket of uneven problems), every
// candidate (Chebyshev order, leaf size, tree kind: uniform or adaptive)
// gets its own tree; its product is
// timed on the device with CUDA events (after a warm-up that builds the
// window caches) and compared with the on-the-fly dense product of the same
// vector.  The fastest candidate whose relative error stays within the
// bound wins; candidates within 3 % of its time count as equally fast and
// the more accurate of them is taken.  The caller builds the bucket's trees with the winner
// (ddm_build_tree_params).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

// max over the three output blocks of max|a - b| / max|b|, on the device:
// per block the two maxima by atomic max on the float bits (non-negative)
__global__ void k_blockmax(const double *a, const double *b, int64_t n, unsigned long long *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int blk = (int)(i / n);
    const double d = fabs(a[i] - b[i]), r = fabs(b[i]);
    atomicMax(&out[2 * blk], (unsigned long long)__double_as_longlong(d));
    atomicMax(&out[2 * blk + 1], (unsigned long long)__double_as_longlong(r));
}

double bits2d(unsigned long long v) {
    double d;
    std::memcpy(&d, &v, sizeof d);
    return d;
}

}  // namespace

extern "C" ddm_status ddm_autotune(ddm_ctx *ctx, const double *d_xy, int64_t n, const double *d_x, double dt,
                                   const int *orders, int n_orders, const int *leaves, int n_leaves,
                                   double max_rel_err, ddm_fmm_params *best, double *best_ms, double *best_err) {
    if (!ctx || !d_xy || !d_x || n <= 0 || !(dt > 0) || !best || !(max_rel_err > 0))
        return ctx_fail(ctx, DDM_EINVAL, "ddm_autotune: bad arguments");
    static const int def_orders[] = {4, 6, 8, 10, 12};
    static const int def_leaves[] = {16, 32, 64};
    if (!orders || n_orders <= 0) { orders = def_orders; n_orders = 5; }
    if (!leaves || n_leaves <= 0) { leaves = def_leaves; n_leaves = 3; }
    cudaStream_t s = ctx->stream;
    double *yd = nullptr, *yf = nullptr;
    unsigned long long *mx = nullptr;
    DDM_CUDA_TRY(ctx, dalloc(&yd, 3 * n * sizeof(double), s));
    DDM_CUDA_TRY(ctx, dalloc(&yf, 3 * n * sizeof(double), s));
    DDM_CUDA_TRY(ctx, dalloc(&mx, 6 * sizeof(unsigned long long), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DDM_CUDA_TRY(ctx, cudaEventCreate(&e0));
    DDM_CUDA_TRY(ctx, cudaEventCreate(&e1));
    ddm_status st = DDM_OK;
    double bms = 1e300, berr = 0.0;
    ddm_fmm_params bp = ctx->prm;
    bool found = false;
    // the reference: the dense product on one candidate's tree (any tree of
    // the geometry gives the same dense product)
    bool have_ref = false;
    const int reps = 5;
    for (int io = 0; io < n_orders && !st; ++io)
        for (int ic = 0; ic < 2 * n_leaves && !st; ++ic) {
            ddm_fmm_params p = ctx->prm;
            p.n_cheb = orders[io];
            p.leaf_size = leaves[ic >> 1];
            p.adaptive = ic & 1;
            p.max_depth = 0;
            if (p.n_cheb < 2 || p.n_cheb > DDM_MAX_CHEB || (p.n_cheb & 1) || p.leaf_size <= 0) continue;
            ddm_tree *t = nullptr;
            if ((st = tree_build(ctx, d_xy, n, p, &t))) break;
            if (!have_ref) {
                if ((st = op_apply(ctx, t, 0.0, dt, d_x, yd, DDM_MODE_DENSE, 0, 1.0))) { tree_free(t); break; }
                have_ref = true;
            }
            // warm-up: workspace, own-element blocks and M2L operators of the window
            if ((st = op_apply(ctx, t, 0.0, dt, d_x, yf, DDM_MODE_FMM, 0, 1.0))) { tree_free(t); break; }
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && !st; ++r) st = op_apply(ctx, t, 0.0, dt, d_x, yf, DDM_MODE_FMM, 0, 1.0);
            cudaEventRecord(e1, s);
            if (st) { tree_free(t); break; }
            cudaMemsetAsync(mx, 0, 6 * sizeof(unsigned long long), s);
            k_blockmax<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(yf, yd, n, mx);
            unsigned long long h[6];
            cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, s);
            cudaError_t ce = cudaStreamSynchronize(s);
            tree_free(t);
            if (ce != cudaSuccess) { st = ctx_fail(ctx, DDM_ECUDA, cudaGetErrorString(ce)); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            double err = 0.0, top = 0.0;
            for (int b = 0; b < 3; ++b) top = std::max(top, bits2d(h[2 * b + 1]));
            for (int b = 0; b < 3; ++b) {
                const double d = bits2d(h[2 * b]), r = bits2d(h[2 * b + 1]);
                // a block that is numerically zero is measured against 1e-4 of the largest
                const double sc = std::max(r, 1e-4 * top);
                if (sc > 0) err = std::max(err, d / sc);
            }
            // within the bound, the fastest; a candidate within 3 % of the
            // best time wins if it is more accurate (timing noise must not
            // pick a lower order whose error the sample does not exercise)
            const bool faster = ms < 0.97 * bms, tie = ms < 1.03 * bms && err < berr;
            if (err <= max_rel_err && (!found || faster || tie)) {
                bms = ms;
                berr = err;
                bp = p;
                found = true;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(yd, s);
    dfree(yf, s);
    dfree(mx, s);
    if (st) return st;
    if (!found) return ctx_fail(ctx, DDM_ENOTCONV, "ddm_autotune: no candidate within the error bound");
    *best = bp;
    if (best_ms) *best_ms = bms;
    if (best_err) *best_err = berr;
    return DDM_OK;
}
