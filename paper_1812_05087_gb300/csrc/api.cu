// C ABI of the library: context, tree handles, products, history sum,
// right-hand side, GMRES (FP64, device-resident Krylov basis) and SIFs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

ddm_status ctx_fail(ddm_ctx *ctx, ddm_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

void prof_begin(ddm_ctx *ctx, int stage) {
    if (!ctx->prof.on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, ctx->stream);
    ctx->prof.open_stage = stage;
    ctx->prof.open_ev = e;
}
void prof_end(ddm_ctx *ctx, int stage, int launches) {
    ctx->prof.launches[stage] += launches;
    if (!ctx->prof.on || ctx->prof.open_stage != stage) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, ctx->stream);
    ctx->prof.ev.push_back({stage, {ctx->prof.open_ev, e}});
    ctx->prof.open_stage = -1;
}

namespace {

// S_n(xi_a, x): Chebyshev cardinal function at the roots of T_n (paper Sec. 3.2)
double cheb_S(int n, double xa, double x) {
    double s = 1.0 / n, t0a = 1, t1a = xa, t0 = 1, t1 = x;
    for (int k = 1; k < n; ++k) {
        s += 2.0 / n * t1a * t1;
        double t2a = 2 * xa * t1a - t0a, t2 = 2 * x * t1 - t0;
        t0a = t1a; t1a = t2a; t0 = t1; t1 = t2;
    }
    return s;
}

ddm_status valid_material(const ddm_material *m) {
    if (!m) return DDM_EINVAL;
    if (!(m->G > 0) || !(m->nu >= 0) || !(m->nu < m->nu_u) || !(m->nu_u < 0.5) || !(m->B > 0) || !(m->B <= 1) ||
        !(m->perm > 0) || !(m->visc > 0))
        return DDM_EINVAL;
    return DDM_OK;
}

// ------------------------------------------------------------- small kernels
__global__ void k_rhs(const double *xy, int64_t n, ddm_loads L, const double *pf, double *b) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double dx = xy[2 * n + e] - xy[e], dy = xy[3 * n + e] - xy[n + e];
    double len = hypot(dx, dy), tx = dx / len, ty = dy / len, nx = -ty, ny = tx;
    double sxx = -L.sigma_H, syy = -L.sigma_h;            // tension positive far field
    double snn = sxx * nx * nx + syy * ny * ny, tau = sxx * tx * nx + syy * ty * ny;
    double p_f = pf ? pf[e] : L.p_f;
    b[e] = -tau;
    b[n + e] = (L.system == DDM_SYS_RATE) ? (-L.p0 - snn) : (-p_f - snn);
    b[2 * n + e] = (L.system == DDM_SYS_PRESSURE) ? (p_f - L.p0) : 0.0;
}

__global__ void k_sif(const double *xy, int64_t n, const double *x, const int64_t *tip, int m, double G, double nu,
                      double *KI, double *KII) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t e = tip[i];
    double a = 0.5 * hypot(xy[2 * n + e] - xy[e], xy[3 * n + e] - xy[n + e]);
    double E = 2.0 * G * (1.0 + nu);
    double f = 0.806 * E / (4.0 * (1.0 - nu * nu)) * sqrt(M_PI / (2.0 * a));
    KI[i] = f * x[n + e];
    KII[i] = f * x[e];
}

// --- GMRES helpers (FP64).  Reduced vectors (length nu) live in the first
// ncomp blocks of N of a 3N vector layout.
// Dot products h[v] = V[v] . w for all v < nv in two steps without atomics:
// every block covers one contiguous chunk of the vectors, each thread
// carrying up to DP_V partial sums in registers, reduced across the warp by
// shuffles and across the block in shared memory into part[block][v]; the
// final kernel sums the blocks (one warp per vector) and maintains the
// Hessenberg column (hcol = h on the first CGS pass, += h on the second).
constexpr int DP_T = 128, DP_V = 8, DP_G = 304;
__global__ void __launch_bounds__(DP_T) k_dots_part(const double *V, int64_t ld, int nv, const double *w, int64_t len,
                                                    int64_t chunk, double *part, int pld) {
    __shared__ double red[DP_T / 32][DP_V];
    const int64_t i0 = blockIdx.x * chunk, i1 = i0 + chunk < len ? i0 + chunk : len;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int v0 = 0; v0 < nv; v0 += DP_V) {
        double acc[DP_V];
#pragma unroll
        for (int q = 0; q < DP_V; ++q) acc[q] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += DP_T) {
            const double wi = w[i];
#pragma unroll
            for (int q = 0; q < DP_V; ++q)
                if (v0 + q < nv) acc[q] = fma(V[(int64_t)(v0 + q) * ld + i], wi, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < DP_V; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xFFFFFFFFu, acc[q], o);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < DP_V; ++q) red[wid][q] = acc[q];
        __syncthreads();
        if (threadIdx.x < DP_V && v0 + threadIdx.x < nv) {
            double sum = 0.0;
#pragma unroll
            for (int k = 0; k < DP_T / 32; ++k) sum += red[k][threadIdx.x];
            part[(int64_t)blockIdx.x * pld + v0 + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}
__global__ void k_dots_final(const double *part, int G, int pld, int nv, double *h, double *hcol, int accumulate) {
    const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (v >= nv) return;
    double sum = 0.0;
    for (int b = lane; b < G; b += 32) sum += part[(int64_t)b * pld + v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    if (lane == 0) {
        h[v] = sum;
        if (hcol) hcol[v] = accumulate ? hcol[v] + sum : sum;
    }
}
// One Arnoldi orthogonalisation step as a single cooperative kernel, one
// block per SM (its blocks meet at grid barriers, so it is launched
// cooperatively, which guarantees they are all resident).  A pass:
//   1. partial dot products of w with V[0..nv) and with itself over the
//      block's chunk (warp q takes vectors q, q + OR_W, ...);   barrier
//   2. every block sums all partials itself, in the same order, so h and
//      ||w||^2 are identical everywhere (block 0 records hcol = or += h);
//      w -= V h on the chunk;
//   3. ||w_new||^2 = ||w||^2 - |h|^2 (V orthonormal) and the
//      Daniel-Gragg-Kaufman-Stewart decision, the same in every block: a
//      second pass when ||w_new||^2 < |h|^2, i.e. when more than half of
//      ||w||^2 was removed.  Without a second pass the difference keeps at
//      least half of ||w||^2, so it is accurate to a few rounding units; in
//      the second pass h is small against the explicit ||w||^2.
// Then V[nv] = w / ||w||, hcol[nv] = ||w||: one grid barrier per pass.  The
// partials are stored by vector (part[v G + block]) for coalesced sums, each
// pass in its own half of part[] (2 (nv + 1) G doubles).  The
// barriers give up after max_polls polls (ddm_set_wait_limit) and raise the
// error word (the results are then invalid, nothing hangs; the solve that
// reads the word resets the barrier counters).
__device__ __forceinline__ void grid_barrier(unsigned *bar, int *err, long long max_polls) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vb = bar;
        const unsigned gen = vb[1];
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            long long polls = 0;
            while (vb[1] == gen) {
                if (++polls > max_polls) { atomicExch(err, 1); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}
constexpr int OR_T = 512, OR_W = OR_T / 32;
__global__ void __launch_bounds__(OR_T) k_arnoldi_orth(double *V, int64_t len, int nv, double *w, int64_t chunk,
                                                       double *part, double *hcol, unsigned *bar, int *err,
                                                       long long max_polls) {
    __shared__ double sh[512 + 1];
    __shared__ double s_hh;
    const int64_t i0 = blockIdx.x * chunk, i1 = i0 + chunk < len ? i0 + chunk : len;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x;
    double nrm2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        // each pass its own partials: a block may start the second pass while
        // another still sums the first pass's
        double *pp = part + (int64_t)pass * (nv + 1) * G;
        // 1. partial dots; vector nv is w itself
        for (int v = wid; v <= nv; v += OR_W) {
            const double *Vv = v < nv ? V + (int64_t)v * len : w;
            double acc = 0.0;
            for (int64_t i = i0 + lane; i < i1; i += 32) acc = fma(Vv[i], w[i], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (lane == 0) pp[(int64_t)v * G + blockIdx.x] = acc;
        }
        grid_barrier(bar, err, max_polls);
        // 2. h and ||w||^2 (every block, same order)
        for (int v = wid; v <= nv; v += OR_W) {
            double sum = 0.0;
            for (int b = lane; b < G; b += 32) sum += __ldcg(pp + (int64_t)v * G + b);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
            if (lane == 0) sh[v] = sum;
        }
        __syncthreads();
        if (wid == 0) {
            double hh = 0.0;
            for (int v = lane; v < nv; v += 32) hh = fma(sh[v], sh[v], hh);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hh += __shfl_xor_sync(0xFFFFFFFFu, hh, o);
            if (lane == 0) s_hh = hh;
        }
        if (blockIdx.x == 0)
            for (int v = tid; v < nv; v += OR_T) hcol[v] = pass ? hcol[v] + sh[v] : sh[v];
        for (int64_t i = i0 + tid; i < i1; i += OR_T) {
            double sum = 0.0;
            for (int v = 0; v < nv; ++v) sum = fma(sh[v], V[(int64_t)v * len + i], sum);
            w[i] -= sum;
        }
        __syncthreads();                      // s_hh written; w updated before the next pass reads it
        // 3. norm and the second-pass decision
        const double hh = s_hh, rest = sh[nv] - hh;
        nrm2 = rest > 0.0 ? rest : 0.0;
        if (!(pass == 0 && rest < hh)) break;
        __syncthreads();                      // sh is rewritten by the next pass
    }
    // next basis vector
    const double nrm = sqrt(nrm2), inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (blockIdx.x == 0 && tid == 0) hcol[nv] = nrm;
    double *out = V + (int64_t)nv * len;
    for (int64_t i = i0 + tid; i < i1; i += OR_T) out[i] = w[i] * inv;
}
// restrict a 3N product or right-hand side to the system rows (RATE:
// sigma_n + p when combine = 1; a right-hand side carries the p part of a
// subtracted history term in its third block)
__global__ void k_restrict(const double *y, int64_t n, int sys, int combine, double *out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = y[e];
    out[n + e] = y[n + e] + (combine && sys == DDM_SYS_RATE ? y[2 * n + e] : 0.0);
    if (sys == DDM_SYS_PRESSURE) out[2 * n + e] = y[2 * n + e];
}
__global__ void k_axpy(double a, const double *x, double *y, int64_t len) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < len) y[i] += a * x[i];
}
__global__ void k_comb(const double *V, int64_t ld, int nv, const double *yv, double *out, int64_t len) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = 0;
    for (int v = 0; v < nv; ++v) s += yv[v] * V[v * ld + i];
    out[i] = s;
}

inline unsigned nblk(int64_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

}  // namespace

struct GmresWork {
    int64_t cap_len = 0;       // system length (nc N) the basis was sized for
    int64_t cap_n = 0;         // elements the 3N vectors were sized for
    int cap_m = 0;
    cudaStream_t st = nullptr;
    double *V = nullptr, *w = nullptr, *full = nullptr, *y3 = nullptr, *b = nullptr;
    double *hcol = nullptr, *nrm = nullptr, *part = nullptr;
    unsigned *cnt = nullptr;   // grid-barrier counter and generation (zero between launches)
    double *hpin = nullptr;    // pinned host slots: a norm, and per step the least-squares status (2 x 4)
    cudaEvent_t ev[2] = {nullptr, nullptr};   // one per pinned status slot
    LsqDev lsq;                // device least squares (krylov.cu)
    void release() {
        double *ps[] = {V, w, full, y3, b, hcol, nrm, part};
        cudaStream_t s = st;
        for (double *p : ps) dfree(p, s);
        dfree(cnt, s);
        lsq_free(lsq, s);
        if (hpin) cudaFreeHost(hpin);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        *this = GmresWork();
        st = s;
    }
};

extern "C" {

ddm_status ddm_create(ddm_ctx **out, const ddm_material *mat, const ddm_fmm_params *prm, void *cuda_stream) {
    if (!out) return DDM_EINVAL;
    *out = nullptr;
    if (valid_material(mat) != DDM_OK) return DDM_EINVAL;
    ddm_fmm_params p = prm ? *prm : ddm_fmm_params{8, 32, 0, 6, 0};
    if (p.n_cheb <= 0) p.n_cheb = 8;
    if (p.leaf_size <= 0) p.leaf_size = 32;
    if (p.quad_near <= 0) p.quad_near = 6;
    if (p.n_cheb < 2 || p.n_cheb > DDM_MAX_CHEB || (p.n_cheb & 1) || p.quad_near > 16 || p.max_depth < 0 ||
        p.adaptive < 0 || p.adaptive > 2)
        return DDM_EINVAL;
    ddm_ctx *c = new (std::nothrow) ddm_ctx();
    if (!c) return DDM_ENOMEM;
    c->mat = *mat;
    c->prm = p;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return DDM_ECUDA; }
    {   // keep freed pool memory inside the process (stream-ordered reuse)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    const ddm_material &m = *mat;
    double G = m.G, nu = m.nu, nuu = m.nu_u, B = m.B;
    double alpha = 3 * (nuu - nu) / (B * (1 - 2 * nu) * (1 + nuu));
    double eta = alpha * (1 - 2 * nu) / (2 * (1 - nu));
    double M = 2 * G * (nuu - nu) / (alpha * alpha * (1 - 2 * nuu) * (1 - 2 * nu));
    double S = alpha * eta / G + 1 / M;
    double kappa = m.perm / m.visc;
    double kpsi = alpha * eta / (G * S);
    KConst<double> kd;
    kd.G2 = 2 * G;
    kd.Cel = G / (2 * M_PI * (1 - nu));
    kd.Ce = (1 - 2 * nu) / (2 * M_PI * (1 - nu));
    kd.K2 = kpsi * kd.Ce / 4;
    kd.aS = alpha / S;
    kd.eta = eta;
    kd.i4pk = 1 / (4 * M_PI * kappa);
    kd.c = kappa / S;
    kd.Cu = kd.Cel + 2 * kd.G2 * kd.K2;
    kd.pS = kd.aS * kd.Ce;
    kd.a6 = 6 * kd.G2 * kd.K2;
    kd.qe = kd.eta * kd.i4pk;
    c->kd = kd;
    c->kf = KConst<float>{(float)kd.G2, (float)kd.Cel, (float)kd.Ce, (float)kd.K2, (float)kd.aS, (float)kd.eta,
                          (float)kd.i4pk, (float)kd.c, (float)kd.Cu, (float)kd.pS, (float)kd.a6, (float)kd.qe};
    // M2M / L2L transfer matrices T[q][a][a'] = S_n(xi_a, (xi_a' + q)/2)
    // (q = the child's half), for every even order: trees may carry their own
    for (int nn = 2; nn <= DDM_MAX_CHEB; nn += 2) {
        std::vector<double> xn(nn);
        for (int j = 0; j < nn; ++j) xn[j] = cos((2 * j + 1) * M_PI / (2.0 * nn));
        std::vector<float> Tn(2 * nn * nn);
        for (int q = 0; q < 2; ++q)
            for (int a = 0; a < nn; ++a)
                for (int ap = 0; ap < nn; ++ap)
                    Tn[q * nn * nn + a * nn + ap] = (float)cheb_S(nn, xn[a], 0.5 * (xn[ap] + (q ? 1.0 : -1.0)));
        if (cudaMalloc(&c->cheb_Tn[nn / 2 - 1], Tn.size() * sizeof(float)) != cudaSuccess) {
            for (float *p : c->cheb_Tn) if (p) cudaFree(p);
            delete c;
            return DDM_ENOMEM;
        }
        cudaMemcpy(c->cheb_Tn[nn / 2 - 1], Tn.data(), Tn.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        for (float *p : c->cheb_Tn) if (p) cudaFree(p);
        delete c;
        return DDM_ENOMEM;
    }
    {   // auxiliary stream (highest priority: the far field is the longer branch)
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            for (float *p : c->cheb_Tn) if (p) cudaFree(p);
            cudaFree(c->d_err);
            delete c;
            return DDM_ECUDA;
        }
    }
    c->gm = new GmresWork();
    *out = c;
    return DDM_OK;
}

void ddm_destroy(ddm_ctx *ctx) {
    if (!ctx) return;
    for (float *p : ctx->cheb_Tn)
        if (p) cudaFree(p);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
    if (ctx->hist_M) cudaFree(ctx->hist_M);
    if (ctx->hist_C) cudaFree(ctx->hist_C);
    if (ctx->gm) { ctx->gm->release(); delete ctx->gm; }
    delete ctx;
}

const char *ddm_last_error(const ddm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ddm_status ddm_device_check(ddm_ctx *ctx) {
    if (!ctx) return DDM_EINVAL;
    int h = 0;
    DDM_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (!h) return DDM_OK;
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    return ctx_fail(ctx, DDM_ETIMEOUT, "a bounded device wait expired (results of the affected calls are invalid)");
}

ddm_status ddm_set_wait_limit(ddm_ctx *ctx, int64_t polls) {
    if (!ctx || polls < 0) return ctx_fail(ctx, DDM_EINVAL, "ddm_set_wait_limit: bad arguments");
    ctx->grid_polls = polls == 0 ? (1ll << 22) : (long long)polls;
    return DDM_OK;
}

ddm_status ddm_set_m2l_compression(ddm_ctx *ctx, int mode, int rank) {
    if (!ctx || mode < 0 || mode > 2 || rank < 0 || rank > 512 || rank % 8)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_set_m2l_compression: mode 0, 1 or 2; rank 0 or a multiple of 8 up to 512");
    ctx->m2l_compress = mode;
    ctx->m2l_rank = rank;
    return DDM_OK;
}

ddm_status ddm_profile(ddm_ctx *ctx, int enable) {
    if (!ctx) return DDM_EINVAL;
    ctx->prof.on = enable ? 1 : 0;
    return DDM_OK;
}

ddm_status ddm_profile_read(ddm_ctx *ctx, double *ms, int64_t *launches) {
    if (!ctx || !ms || !launches) return DDM_EINVAL;
    DDM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < DDM_NSTAGES; ++k) { ms[k] = 0.0; launches[k] = ctx->prof.launches[k]; ctx->prof.launches[k] = 0; }
    for (auto &p : ctx->prof.ev) {
        float t = 0.f;
        cudaEventElapsedTime(&t, p.second.first, p.second.second);
        ms[p.first] += t;
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    ctx->prof.ev.clear();
    return DDM_OK;
}

ddm_status ddm_build_tree(ddm_ctx *ctx, const double *d_xy, int64_t n, ddm_tree **out) {
    if (!ctx) return DDM_EINVAL;
    return tree_build(ctx, d_xy, n, ctx->prm, out);
}

ddm_status ddm_build_tree_params(ddm_ctx *ctx, const double *d_xy, int64_t n, const ddm_fmm_params *prm,
                                 ddm_tree **out) {
    if (!ctx) return DDM_EINVAL;
    if (!prm) return tree_build(ctx, d_xy, n, ctx->prm, out);
    ddm_fmm_params p = *prm;
    if (p.n_cheb <= 0) p.n_cheb = ctx->prm.n_cheb;
    if (p.leaf_size <= 0) p.leaf_size = ctx->prm.leaf_size;
    if (p.quad_near <= 0) p.quad_near = ctx->prm.quad_near;
    if (p.n_cheb < 2 || p.n_cheb > DDM_MAX_CHEB || (p.n_cheb & 1) || p.quad_near > 16 || p.max_depth < 0 ||
        p.adaptive < 0 || p.adaptive > 2)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_build_tree_params: bad FMM parameters");
    return tree_build(ctx, d_xy, n, p, out);
}

void ddm_tree_destroy(ddm_tree *tree) { tree_free(tree); }

ddm_status ddm_tree_get_info(const ddm_tree *t, ddm_tree_info *info) {
    if (!t || !info) return DDM_EINVAL;
    info->n_elements = t->n;
    info->depth = t->depth;
    info->n_cells = t->n_cells;
    info->n_leaves = t->n_leaf;
    info->n_m2l_pairs = t->n_m2l;
    info->n_p2p_pairs = t->n_p2p;
    info->root_half_width = t->h0;
    info->leaf_level_min = t->leaf_level_min;
    info->adaptive = t->adaptive;
    info->max_leaf_records = t->max_recs;
    return DDM_OK;
}

ddm_status ddm_matvec(ddm_ctx *ctx, const ddm_tree *tree, double tau_lo, double tau_hi, const double *d_x, double *d_y,
                      int mode) {
    int base = mode & ~DDM_MODE_PRECISE;
    if (!ctx || !tree || !d_x || !d_y || d_x == d_y || (base != DDM_MODE_FMM && base != DDM_MODE_DENSE))
        return ctx_fail(ctx, DDM_EINVAL, "ddm_matvec: bad arguments");
    return op_apply(ctx, const_cast<ddm_tree *>(tree), tau_lo, tau_hi, d_x, d_y, mode, 0, 1.0);
}

ddm_status ddm_history_apply(ddm_ctx *ctx, const ddm_tree *tree, const double *d_hist, const double *h_times, int H,
                             double *d_rhs, int mode) {
    if (!ctx || !tree || H < 0 || (H > 0 && (!d_hist || !h_times)) || !d_rhs)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_history_apply: bad arguments");
    if (H == 0) return DDM_OK;
    for (int k = 0; k <= H; ++k)
        if (!(h_times[k + 1] > h_times[k])) return ctx_fail(ctx, DDM_EINVAL, "ddm_history_apply: times must increase");
    ddm_tree *t = const_cast<ddm_tree *>(tree);
    if (ctx->hist_E > 0 && H > ctx->hist_E) return history_compressed(ctx, t, d_hist, h_times, H, d_rhs, mode);
    int64_t N = t->n;
    double tobs = h_times[H + 1];
    for (int eta = 1; eta <= H; ++eta) {
        double lo = tobs - h_times[eta], hi = tobs - h_times[eta - 1];
        ddm_status st = op_apply(ctx, t, lo, hi, d_hist + (int64_t)(eta - 1) * 3 * N, d_rhs, mode, 1, -1.0);
        if (st) return st;
    }
    return DDM_OK;
}

ddm_status ddm_rhs(ddm_ctx *ctx, const ddm_tree *tree, const ddm_loads *loads, const double *d_pf, double *d_rhs) {
    if (!ctx || !tree || !loads || !d_rhs || loads->system < 0 || loads->system > 2)
        return ctx_fail(ctx, DDM_EINVAL, "ddm_rhs: bad arguments");
    k_rhs<<<nblk(tree->n), 256, 0, ctx->stream>>>(tree->xy_caller, tree->n, *loads, d_pf, d_rhs);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

ddm_status ddm_sif(ddm_ctx *ctx, const ddm_tree *tree, const double *d_x, const int64_t *d_tip, int n, double *d_KI,
                   double *d_KII) {
    if (!ctx || !tree || !d_x || n < 0 || (n > 0 && (!d_tip || !d_KI || !d_KII)))
        return ctx_fail(ctx, DDM_EINVAL, "ddm_sif: bad arguments");
    if (n == 0) return DDM_OK;
    k_sif<<<nblk(n), 256, 0, ctx->stream>>>(tree->xy_caller, tree->n, d_x, d_tip, n, ctx->mat.G, ctx->mat.nu, d_KI,
                                            d_KII);
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return DDM_OK;
}

ddm_status ddm_gmres_solve(ddm_ctx *ctx, const ddm_tree *tree, double dt, const double *d_rhs, double *d_x,
                           const ddm_gmres_params *prm, ddm_gmres_info *info) {
    if (!ctx || !tree || !d_rhs || !d_x || !(dt > 0)) return ctx_fail(ctx, DDM_EINVAL, "ddm_gmres_solve: bad arguments");
    ddm_gmres_params P = prm ? *prm : ddm_gmres_params{DDM_SYS_PRESSURE, 50, 1000, 1e-6, DDM_MODE_FMM};
    if (P.restart <= 0) P.restart = 50;
    if (P.max_iters <= 0) P.max_iters = 1000;
    if (!(P.tol > 0)) P.tol = 1e-6;
    if (P.system < 0 || P.system > 2 || P.restart > 500) return ctx_fail(ctx, DDM_EINVAL, "ddm_gmres_solve: bad params");
    ddm_tree *t = const_cast<ddm_tree *>(tree);
    cudaStream_t s = ctx->stream;
    int64_t N = t->n;
    int nc = P.system == DDM_SYS_PRESSURE ? 3 : 2;
    int64_t len = nc * N;
    int m = P.restart;
    GmresWork &g = *ctx->gm;
    ddm_status st0;
    if (g.cap_len < len || g.cap_n < N || g.cap_m < m) {
        g.release();
        size_t v3 = 3 * N * sizeof(double);
        g.st = s;
        bool ok = dalloc(&g.V, (size_t)(m + 1) * len * sizeof(double), s) == cudaSuccess &&
                  dalloc(&g.w, v3, s) == cudaSuccess &&
                  dalloc(&g.full, v3, s) == cudaSuccess && dalloc(&g.y3, v3, s) == cudaSuccess &&
                  dalloc(&g.b, v3, s) == cudaSuccess &&
                  dalloc(&g.hcol, (m + 2) * sizeof(double), s) == cudaSuccess &&
                  dalloc(&g.nrm, sizeof(double), s) == cudaSuccess &&
                  dalloc(&g.part, (size_t)2 * DP_G * (m + 2) * sizeof(double), s) == cudaSuccess &&
                  dalloc(&g.cnt, 4 * sizeof(unsigned), s) == cudaSuccess &&
                  cudaMemsetAsync(g.cnt, 0, 4 * sizeof(unsigned), s) == cudaSuccess &&
                  cudaMallocHost(&g.hpin, 12 * sizeof(double)) == cudaSuccess &&
                  cudaEventCreateWithFlags(&g.ev[0], cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&g.ev[1], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) { g.release(); return ctx_fail(ctx, DDM_ENOMEM, "GMRES workspace allocation failed"); }
        g.cap_len = len; g.cap_n = N; g.cap_m = m;
    }
    if ((st0 = lsq_alloc(ctx, g.lsq, 1, m, s))) return st0;
    int mode = P.mode & ~DDM_MODE_PRECISE, sys = P.system;
    ddm_status st;
    // operator y(len) = restrict(A(dt) [v; 0]) ; the 3N layout keeps blocks of N
    auto apply = [&](const double *v, double *out, int md) -> ddm_status {
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(g.full, 0, 3 * N * sizeof(double), s));
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(g.full, v, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
        ddm_status e = op_apply(ctx, t, 0.0, dt, g.full, g.y3, md, 0, 1.0);
        if (e) return e;
        k_restrict<<<nblk(N), 256, 0, s>>>(g.y3, N, sys, 1, out);
        return DDM_OK;
    };
    const int pld = m + 2;
    const int64_t chunk = (len + DP_G - 1) / DP_G;
    // cooperative orthogonalisation grid: every block resident at once
    int orth_grid = DP_G;
    {
        int per_sm = 0, nsm = 0;
        DDM_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi_orth, OR_T, 0));
        DDM_CUDA_TRY(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
        if (per_sm < 1) return ctx_fail(ctx, DDM_ECUDA, "ddm_gmres_solve: orthogonalisation kernel cannot be resident");
        orth_grid = std::max(1, std::min(DP_G, nsm));
    }
    const int64_t orth_chunk = (len + orth_grid - 1) / orth_grid;
    // h[v] = V[v] . w, v < nv (hcol: see k_dots_final)
    auto dots = [&](const double *Vb, int nv, const double *w, double *h, double *hcol, int accumulate) {
        k_dots_part<<<DP_G, DP_T, 0, s>>>(Vb, len, nv, w, len, chunk, g.part, pld);
        k_dots_final<<<(nv + 3) / 4, 128, 0, s>>>(g.part, DP_G, pld, nv, h, hcol, accumulate);
    };
    auto norm = [&](const double *v, double &out) -> ddm_status {
        dots(v, 1, v, g.nrm, nullptr, 0);
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(g.hpin, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
        DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        out = sqrt(g.hpin[0]);
        return DDM_OK;
    };
    // preconditioner: inverted chain blocks of this (dt, system)
    if ((st = pb_prepare(ctx, t, dt, sys, s))) return st;
    // b = restrict(rhs) - restrict(A [0; 0; Dq]) for the 2N systems
    k_restrict<<<nblk(N), 256, 0, s>>>(d_rhs, N, sys, 1, g.b);   // RATE: sigma_n + p rows of the RHS
    if (sys != DDM_SYS_PRESSURE) {
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(g.full, 0, 2 * N * sizeof(double), s));
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(g.full + 2 * N, d_x + 2 * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if ((st = op_apply(ctx, t, 0.0, dt, g.full, g.y3, mode | DDM_MODE_PRECISE, 0, 1.0))) return st;
        k_restrict<<<nblk(N), 256, 0, s>>>(g.y3, N, sys, 1, g.w);
        k_axpy<<<nblk(len), 256, 0, s>>>(-1.0, g.w, g.b, len);
    }
    double bnorm, xnorm;
    if ((st = norm(g.b, bnorm))) return st;
    if (bnorm == 0) bnorm = 1;
    if ((st = norm(d_x, xnorm))) return st;     // a zero initial guess needs no product
    bool x_zero = xnorm == 0.0;
    int iters = 0, restarts = 0;
    double rel = 1e300;
    bool conv = false, timed_out = false;
    double best = 1e300;
    int stall = 0;
    // Precision escalates only when a restart cycle stalls (the residual
    // falls by less than 10%): level 0 is plain restarted GMRES with the
    // requested products (paper Sec. 4); level 1 recomputes the residuals
    // with the precise products (mixed-precision refinement, inner solves
    // two decades at a time; residual_mode); level 2 also makes the Arnoldi
    // products precise; level 3 (at most EXACT_OP_MAX elements) takes the
    // exact FP64 dense product for them; three more stalls end the solve.  Long
    // fractures, whose element contributions cancel strongly, are what reach
    // the higher levels.
    int level = 0;
    const int mode0 = mode;
    if ((st = lsq_reset_iters(ctx, g.lsq, s))) return st;
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(g.cnt, 0, 4 * sizeof(unsigned), s));   // grid barrier starts at zero
    while (iters < P.max_iters) {
        // r = b - A x
        if (x_zero) {
            DDM_CUDA_TRY(ctx, cudaMemsetAsync(g.w, 0, len * sizeof(double), s));
            x_zero = false;
        } else {
            if ((st = apply(d_x, g.w, residual_mode(mode0, level, N)))) return st;
        }
        k_axpy<<<nblk(len), 256, 0, s>>>(-1.0, g.b, g.w, len);          // w = A x - b
        double beta;
        if ((st = norm(g.w, beta))) return st;
        rel = beta / bnorm;
        if (rel < P.tol) { conv = true; break; }
        if (rel < 0.9 * best) { best = rel; stall = 0; }
        else if (level < max_level(N)) {
            mode = arnoldi_mode(mode0, ++level, N);
            stall = 0;
            if (level == 1) {             // re-measure with the precise residual first
                best = 1e300;
                continue;
            }
        }
        else if (++stall >= 3) break;
        // inner target: the tolerance, or (refinement) two decades below beta
        double inner = level == 0 ? 0.3 * P.tol * bnorm : std::max(0.3 * P.tol * bnorm, 1e-4 * beta);
        // v0 = -w / beta; g = (beta, 0, ...) on the device
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(g.V, 0, len * sizeof(double), s));
        k_axpy<<<nblk(len), 256, 0, s>>>(-1.0 / beta, g.w, g.V, len);
        if ((st = lsq_begin(ctx, g.lsq, 1, &beta, &inner, nullptr, s))) return st;
        // One Arnoldi step: preconditioner, product, orthogonalisation (V[jj+1],
        // Hessenberg column jj), the Givens step on the device, then the
        // status triple (live, |g_{jj+1}|, error word) into pinned slot jj % 2
        // and its event.  Steps only depend on each other through the device,
        // so step j + 1 is enqueued before the host reads the status of step
        // j: the GPU never waits for the host, and a cycle that ends at
        // column j leaves one discarded step behind (its Givens step sees the
        // problem no longer live and changes nothing).
        auto step = [&](int jj) -> ddm_status {
            double *vj = g.V + (int64_t)jj * len;
            prof_begin(ctx, 8);
            ddm_status e = pb_apply(ctx, t, sys, vj, g.full, s);
            if (e) return e;
            if (sys == DDM_SYS_PRESSURE) {        // the 3N product is already the system's rows
                if ((e = op_apply(ctx, t, 0.0, dt, g.full, g.w, mode, 0, 1.0))) return e;
            } else {
                if ((e = op_apply(ctx, t, 0.0, dt, g.full, g.y3, mode, 0, 1.0))) return e;
                k_restrict<<<nblk(N), 256, 0, s>>>(g.y3, N, sys, 1, g.w);
            }
            // orthogonalise against V[0..jj] and normalise (one cooperative kernel)
            prof_begin(ctx, 8);
            {
                double *Vp = g.V, *wp = g.w, *pp = g.part, *hcp = g.hcol;
                int nvj = jj + 1;
                int64_t ln = len, ch = orth_chunk;
                unsigned *bp = g.cnt;
                int *ep = ctx->d_err;
                long long polls = ctx->grid_polls;
                void *args[] = {&Vp, &ln, &nvj, &wp, &ch, &pp, &hcp, &bp, &ep, &polls};
                DDM_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void *)k_arnoldi_orth, dim3(orth_grid), dim3(OR_T),
                                                              args, 0, s));
            }
            if ((e = lsq_step(ctx, g.lsq, 1, g.hcol, m + 2, jj, P.max_iters, false, true, s))) return e;
            prof_end(ctx, 8, 2);      // orthogonalisation + Givens step
            DDM_CUDA_TRY(ctx, cudaMemcpyAsync(g.hpin + 4 + (jj & 1) * 4, g.lsq.stat, 3 * sizeof(double),
                                              cudaMemcpyDeviceToHost, s));
            DDM_CUDA_TRY(ctx, cudaEventRecord(g.ev[jj & 1], s));
            return DDM_OK;
        };
        int j = 0;
        bool pending = j < m && iters < P.max_iters;
        if (pending && (st = step(0))) return st;
        while (pending) {
            const bool more = j + 1 < m && iters + 1 < P.max_iters;
            if (more && (st = step(j + 1))) return st;
            DDM_CUDA_TRY(ctx, cudaEventSynchronize(g.ev[j & 1]));
            const double *stat = g.hpin + 4 + (j & 1) * 4;
            rel = stat[1] / bnorm;
            ++j;
            ++iters;
            if (stat[2] != 0.0) { timed_out = true; break; }
            if (stat[0] == 0.0) break;
            pending = more;
        }
        if (timed_out) break;
        // least squares on the device (y = R^-1 g), x += M^-1 V y
        if (j > 0) {
            if ((st = lsq_solve(ctx, g.lsq, 1, s))) return st;
            k_comb<<<nblk(len), 256, 0, s>>>(g.V, len, j, g.lsq.y, g.w, len);
            if ((st = pb_apply(ctx, t, sys, g.w, g.full, s))) return st;
            k_axpy<<<nblk(len), 256, 0, s>>>(1.0, g.full, d_x, len);
        }
        ++restarts;
    }
    if (timed_out) {
        // a grid barrier gave up: the solve's results are invalid; the
        // barrier counters and the error word are reset after the work
        // already enqueued, so that the context stays usable
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(g.cnt, 0, 4 * sizeof(unsigned), s));
        DDM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
        DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (info) {
            info->iterations = iters;
            info->restarts = restarts;
            info->rel_residual = rel;
            info->converged = 0;
        }
        return ctx_fail(ctx, DDM_ETIMEOUT, "ddm_gmres_solve: a bounded device wait expired (the solution is invalid)");
    }
    if (info) {
        info->iterations = iters;
        info->restarts = restarts;
        info->rel_residual = rel;
        info->converged = conv ? 1 : 0;
    }
    DDM_CUDA_TRY(ctx, cudaGetLastError());
    return conv ? DDM_OK : ctx_fail(ctx, DDM_ENOTCONV, "GMRES did not converge");
}

}  // extern "C"
