// Time-compressed history sum (an extension of the paper's time marching,
// Sec. 4: the history of all previous steps is subtracted at every step).
//
// The history at t_obs = t_{H+1} is  sum_{eta=1..H} W(lo_eta, hi_eta) D^eta,
// W(lo, hi) = A(hi) - A(lo), lo_eta = t_obs - t_eta, hi_eta = t_obs - t_{eta-1}:
// one FMM product per past step, O(H^2) products over a march.  The
// response A(tau) is analytic in s = log tau in a strip around the real
// axis (its transient parts are functions of r^2 / (4 c tau), entire in s
// apart from a term linear in s), so over a block of past steps whose
// windows lie in [a, b] with b / a bounded, Chebyshev interpolation in s at
// p nodes alpha_m is accurate to the p-th power of a fixed ratio:
//     A(tau) ~ sum_m A(alpha_m) l_m(log tau),
//     sum_{eta in block} W(lo_eta, hi_eta) D^eta ~ sum_m A(alpha_m) M_m,
//     M_m = sum_eta [l_m(log hi_eta) - l_m(log lo_eta)] D^eta.
// The Lagrange weights sum to one, so sum_m M_m = 0 and the block equals
// sum_{m != m*} [A(alpha_m) - A(alpha_m*)] M_m: p - 1 window products with
// alpha_m* the largest node, and no instantaneous (elastic) part, which
// cancels exactly.  The E most recent steps stay exact; older steps fall
// into blocks [tau_E rho^b, tau_E rho^(b+1)) by lo_eta (tau_E: lo of the
// newest compressed step), each interpolated over [tau_E rho^b,
// tau_E rho^(b+1) (1 + 1/E)] (widened if a window reaches further), so that
// with a constant step the nodes, and hence the cached window operators,
// are the same at every step.  Products per step: E + (p - 1) log_rho(H / E)
// instead of H.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "internal.h"

namespace {

constexpr int HP_MAX = 16;

// M_m[e] = sum_k C[m nb + k] D[(k0 + k) len + e], m < p (FP64)
__global__ void k_hist_moments(const double *D, int64_t len, int k0, int nb, const double *C, int p, double *M) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= len) return;
    double acc[HP_MAX];
#pragma unroll
    for (int m = 0; m < HP_MAX; ++m) acc[m] = 0.0;
    for (int k = 0; k < nb; ++k) {
        const double d = D[(int64_t)(k0 + k) * len + e];
#pragma unroll
        for (int m = 0; m < HP_MAX; ++m)
            if (m < p) acc[m] = fma(C[m * nb + k], d, acc[m]);
    }
#pragma unroll
    for (int m = 0; m < HP_MAX; ++m)
        if (m < p) M[(int64_t)m * len + e] = acc[m];
}

// Lagrange basis of the nodes s[0..p) at x
void lagrange(const double *s, int p, double x, double *l) {
    for (int m = 0; m < p; ++m) {
        double v = 1.0;
        for (int q = 0; q < p; ++q)
            if (q != m) v *= (x - s[q]) / (s[m] - s[q]);
        l[m] = v;
    }
}

// log tau rounded to a 2^-24 grid (down or up): the block ends of steps that
// differ by rounding of t_obs - t_eta land on the same cached windows
double snap_log(double x, bool up) {
    const double q = 16777216.0;
    return (up ? std::ceil(x * q) : std::floor(x * q)) / q;
}

}  // namespace

extern "C" ddm_status ddm_set_history_compression(ddm_ctx *ctx, int exact_steps, int nodes, double ratio) {
    if (!ctx || exact_steps < 0 || (exact_steps > 0 && (nodes < 2 || nodes > HP_MAX || !(ratio >= 1.5) || ratio > 16.0)))
        return ctx_fail(ctx, DDM_EINVAL,
                        "ddm_set_history_compression: exact_steps >= 0; nodes 2..16 and ratio in [1.5, 16] when on");
    ctx->hist_E = exact_steps;
    ctx->hist_p = nodes;
    ctx->hist_rho = ratio;
    return DDM_OK;
}

ddm_status history_compressed(ddm_ctx *ctx, ddm_tree *t, const double *d_hist, const double *h_times, int H,
                              double *d_rhs, int mode) {
    const int E = ctx->hist_E, p = ctx->hist_p;
    const double rho = ctx->hist_rho;
    const int64_t len = 3 * t->n;
    const double tobs = h_times[H + 1];
    cudaStream_t s = ctx->stream;
    ddm_status st;
    // the E most recent steps: exact windows
    for (int eta = H - E + 1; eta <= H; ++eta) {
        if ((st = op_apply(ctx, t, tobs - h_times[eta], tobs - h_times[eta - 1], d_hist + (int64_t)(eta - 1) * len,
                           d_rhs, mode, 1, -1.0)))
            return st;
    }
    // blocks of the older steps (eta = 1 .. H - E), each a contiguous range of eta
    const double tauE = tobs - h_times[H - E];
    std::map<int, std::pair<int, int>> blocks;             // b -> (eta_min, eta_max)
    for (int eta = H - E; eta >= 1; --eta) {
        const double lo = tobs - h_times[eta];
        const int b = (int)std::floor(std::log(lo / tauE) / std::log(rho) + 1e-12);
        auto it = blocks.find(b);
        if (it == blocks.end()) blocks[b] = {eta, eta};
        else it->second.first = eta;
    }
    int nbmax = 0;
    for (auto &kv : blocks) nbmax = std::max(nbmax, kv.second.second - kv.second.first + 1);
    if (ctx->hist_M_cap < (int64_t)p * len) {
        dfree(ctx->hist_M, s);
        ctx->hist_M = nullptr;
        DDM_CUDA_TRY(ctx, dalloc(&ctx->hist_M, (size_t)p * len * sizeof(double), s));
        ctx->hist_M_cap = (int64_t)p * len;
    }
    if (ctx->hist_C_cap < (int64_t)p * nbmax) {
        dfree(ctx->hist_C, s);
        ctx->hist_C = nullptr;
        DDM_CUDA_TRY(ctx, dalloc(&ctx->hist_C, (size_t)p * nbmax * sizeof(double), s));
        ctx->hist_C_cap = (int64_t)p * nbmax;
    }
    std::vector<double> C((size_t)p * nbmax), lh(p), ll(p);
    double snode[HP_MAX], alpha[HP_MAX];
    for (auto &kv : blocks) {
        const int b = kv.first, e0 = kv.second.first, e1 = kv.second.second, nb = e1 - e0 + 1;
        double A = tauE * std::pow(rho, b), B = tauE * std::pow(rho, b + 1) * (1.0 + 1.0 / E);
        for (int eta = e0; eta <= e1; ++eta) {
            A = std::min(A, tobs - h_times[eta]);
            B = std::max(B, tobs - h_times[eta - 1]);
        }
        const double la = snap_log(std::log(A), false), lb = snap_log(std::log(B), true);
        int mp = 0;
        for (int m = 0; m < p; ++m) {
            snode[m] = 0.5 * (la + lb) + 0.5 * (lb - la) * std::cos(M_PI * (2 * m + 1) / (2.0 * p));
            alpha[m] = std::exp(snode[m]);
            if (alpha[m] > alpha[mp]) mp = m;
        }
        // weights of step eta = e0 + k: l_m(log hi) - l_m(log lo)
        for (int k = 0; k < nb; ++k) {
            const int eta = e0 + k;
            lagrange(snode, p, std::log(tobs - h_times[eta - 1]), lh.data());
            lagrange(snode, p, std::log(tobs - h_times[eta]), ll.data());
            for (int m = 0; m < p; ++m) C[(size_t)m * nb + k] = lh[m] - ll[m];
        }
        // (pageable source: the copy is staged before the call returns)
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hist_C, C.data(), (size_t)p * nb * sizeof(double),
                                          cudaMemcpyHostToDevice, s));
        k_hist_moments<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(d_hist, len, e0 - 1, nb, ctx->hist_C, p,
                                                                    ctx->hist_M);
        DDM_CUDA_TRY(ctx, cudaGetLastError());
        // history -= block  <=>  rhs += sum_{m != mp} W(alpha_m, alpha_mp) M_m
        for (int m = 0; m < p; ++m) {
            if (m == mp) continue;
            if ((st = op_apply(ctx, t, alpha[m], alpha[mp], ctx->hist_M + (int64_t)m * len, d_rhs, mode, 1, 1.0)))
                return st;
        }
    }
    return DDM_OK;
}
