// Compressed M2L operators (the low-rank compression of black-box FMM
// operators by singular value decomposition, which the paper cites in
// Sec. 3 as the further step of the Chebyshev FMM; the paper itself applies
// the full operators).
//
// For one time window and one tree level, the operators K_o of every cell
// offset o (4 n^2 x 4 n^2 each) share their row and column spaces up to a
// small numerical rank.  After an equilibration of the four components
// (row and column block scales D_out, D_in: the stress rows and the
// pressure row, the potency columns and the fluid-source column differ by
// many orders), a randomized range finder gives orthonormal bases U (left)
// and V (right) of rank k for all offsets of the level together, from the
// wide and the tall stack of the equilibrated operators K~_o = D_out K_o D_in
// and an independent random test matrix per offset and side:
//     U = orth( sum_o K~_o Omega_o ),   V = orth( sum_o K~_o^T Omega'_o ),
// and the cores C_o = U^T K~_o V (k x k).  Then
//     K_o ~ (D_out^-1 U) C_o (V^T D_in^-1),
// so the M2L of a window becomes three grouped products: W'_J = (V^T D_in^-1)
// W_J per source cell (k values), G'_I = sum_J C_o W'_J per interaction
// pair, F_I += (D_out^-1 U) G'_I per target cell.  No power iteration: the
// singular values of these operators fall off exponentially, so k with its
// oversampling captures the range, and in FP32 a power step (which squares
// the spectrum) would lose the directions below the square root of the
// rounding unit.
//
// The set-up runs once per (tree, window), FP32 on the device, every level
// and both sides at once: bases are held transposed (k x 4 n^2, one basis
// vector per row), every product is one launch of a descriptor-batched GEMM
// that applies the component scales to the operators as it loads them, the
// sums over offsets are split per offset and reduced in a fixed order
// (deterministic), and the orthogonalisations of all (level, side) matrices
// run side by side, one CTA each.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

// One product of a batched GEMM: C (M x N, row-major) = A (M x K, row-major)
// op(B), op(B) = B stored K x N (tb = 0) or B^T with B stored N x K (tb = 1).
// With so given, B's stored entry (i, j) is scaled by so[i / n2] * si[j / n2]
// (the component scales of an M2L operator, rows i and columns j).
struct GDesc {
    const float *A, *B;
    float *C;
    const float *so, *si;
    int tb;
};

constexpr int GT = 64, GK = 32, GP = GT + 4;
__global__ void __launch_bounds__(256) k_gemm_desc(int M, int N, int K, int n2, const GDesc *desc) {
    __shared__ __align__(16) float sa[GK][GP];
    __shared__ __align__(16) float sb[GK][GP];
    const GDesc g = desc[blockIdx.z];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
    const int ldb = g.tb ? K : N;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        // A tile, k fastest: a warp reads 32 consecutive entries of one row
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int ii = e / GK, kk = e % GK, r = r0 + ii, k = k0 + kk;
            sa[kk][ii] = (r < M && k < K) ? g.A[(int64_t)r * K + k] : 0.f;
        }
        // B tile, the stored row's entries fastest
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int ii, kk;
            if (g.tb) { ii = e / GK; kk = e % GK; }
            else { kk = e / GT; ii = e % GT; }
            const int c = c0 + ii, k = k0 + kk;
            float v = 0.f;
            if (c < N && k < K) {
                const int i = g.tb ? c : k, j = g.tb ? k : c;
                v = g.B[(int64_t)i * ldb + j];
                if (g.so) v *= g.so[i / n2] * g.si[j / n2];
            }
            sb[kk][ii] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&sa[kk][4 * ty]);
            const float4 b = *reinterpret_cast<const float4 *>(&sb[kk][4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + 4 * ty + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + 4 * tx + j;
            if (c < N) g.C[(int64_t)r * N + c] = acc[i][j];
        }
    }
}

// Y_m = sum_{z = zo[m]}^{zo[m+1]-1} P_z, in order (elems entries each)
__global__ void k_sum_parts(const float *P, const int *zo, int64_t elems, float *Y) {
    const int m = blockIdx.y;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= elems) return;
    float s = 0.f;
    for (int z = zo[m]; z < zo[m + 1]; ++z) s += P[(int64_t)z * elems + e];
    Y[(int64_t)m * elems + e] = s;
}

// Squared norms of the component blocks of the operators of each level slot
// m = blockIdx.y (keys keys[ko[m]] .. keys[ko[m + 1] - 1]): mode 0 per row
// component, mode 1 per column component of the row-scaled operators
// (row scales S[8 m + 0..3]).  nrm[4 m + c] (double) must start at zero.
__global__ void k_block_norms(const float *ops, const int *keys, const int *ko, int n2, int mode, const float *S,
                              double *nrm) {
    const int m = blockIdx.y, ld = 4 * n2;
    const int64_t big = (int64_t)ld * ld, tot = (int64_t)(ko[m + 1] - ko[m]) * big;
    const float *dout = S + 8 * m;
    double l0 = 0.0, l1 = 0.0, l2 = 0.0, l3 = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / big);
        const int64_t rc = e - o * big;
        const int r = (int)(rc / ld), c = (int)(rc % ld);
        float v = ops[(int64_t)keys[ko[m] + o] * big + rc];
        if (mode) v *= dout[r / n2];
        const int comp = mode ? c / n2 : r / n2;
        const double q = (double)v * v;
        l0 += comp == 0 ? q : 0.0;
        l1 += comp == 1 ? q : 0.0;
        l2 += comp == 2 ? q : 0.0;
        l3 += comp == 3 ? q : 0.0;
    }
    double l[4] = {l0, l1, l2, l3};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double v = l[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&nrm[4 * m + c], v);
    }
}
// scale factors from the block norms: S[8 m + off + c] = 1 / sqrt(nrm[4 m + c]) (1 for an empty block)
__global__ void k_scales(const double *nrm, int nl, int off, float *S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * nl) return;
    const int m = i / 4, c = i % 4;
    S[8 * m + off + c] = nrm[i] > 0.0 ? (float)(1.0 / sqrt(nrm[i])) : 1.f;
}
// a fixed pseudo-random test matrix in [-1, 1] (integer hash of the index)
__global__ void k_rand(float *Om, int64_t n, uint32_t seed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
    Om[i] = (float)(h & 0xFFFFFF) * (2.f / 16777216.f) - 1.f;
}

constexpr int OT = 1024, KMAX = 512;

// Euclidean norm of y (rows entries) over the CTA; red: OT / 32 floats
__device__ float block_norm(const float *y, int rows, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float s = 0.f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) s = fmaf(y[r], y[r], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    __syncthreads();                       // red is free (an earlier reader may still hold it)
    if (lane == 0) red[warp] = s;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return sqrtf(t);
}

// Orthonormal rows of every k x rows matrix Y_m = Y + m k rows (one basis
// vector per row, in place, blockIdx.x = m): classical Gram-Schmidt with two
// passes per vector.  A vector that the passes leave with less than 1e-6 of
// its norm (numerical rank below k) is set to zero.
__global__ void __launch_bounds__(OT) k_orth(float *Y, int rows, int k) {
    __shared__ float d[KMAX];
    __shared__ float red[OT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *Ym = Y + (int64_t)blockIdx.x * k * rows;
    for (int j = 0; j < k; ++j) {
        float *y = Ym + (int64_t)j * rows;
        const float n0 = block_norm(y, rows, red);
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = warp; i < j; i += OT / 32) {
                const float *q = Ym + (int64_t)i * rows;
                float s = 0.f;
                for (int r = lane; r < rows; r += 32) s = fmaf(q[r], y[r], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                if (lane == 0) d[i] = s;
            }
            __syncthreads();
            for (int r = threadIdx.x; r < rows; r += OT) {
                float v = y[r];
                for (int i = 0; i < j; ++i) v = fmaf(-d[i], Ym[(int64_t)i * rows + r], v);
                y[r] = v;
            }
            __syncthreads();
        }
        const float nr = block_norm(y, rows, red);
        // a vector left with less than 1e-6 of its norm lies in the span of
        // the earlier ones to working precision: dropped
        const float inv = (nr > 1e-6f * n0 && nr > 1e-30f) ? 1.f / nr : 0.f;
        for (int r = threadIdx.x; r < rows; r += OT) y[r] *= inv;
        __syncthreads();
    }
}

// per level slot m = blockIdx.y (tree level lvl[m]): pre-operator
// V^T D_in^-1 (k x ld) and post-operator D_out^-1 U (ld x k) from the
// transposed bases Vt = Y_m, Ut = Y_{nl + m}
__global__ void k_pre_post(const float *Y, int nl, const float *S, const int *lvl, int n2, int k, float *pre,
                           float *post) {
    const int m = blockIdx.y, ld = 4 * n2, l = lvl[m];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)ld * k) return;
    const int j = (int)(i / ld), c = (int)(i % ld);      // j: rank index, c: expansion entry
    const float vt = Y[(int64_t)m * k * ld + i], ut = Y[(int64_t)(nl + m) * k * ld + i];
    pre[(int64_t)l * k * ld + i] = vt / S[8 * m + 4 + c / n2];
    post[(int64_t)l * ld * k + (int64_t)c * k + j] = ut / S[8 * m + c / n2];
}

inline dim3 ggrid(int M, int N, int batch) {
    return dim3((unsigned)((N + GT - 1) / GT), (unsigned)((M + GT - 1) / GT), (unsigned)batch);
}

}  // namespace

int svd_rank(const ddm_ctx *ctx, int n) {
    if (n < 8) return 0;                 // 4 n^2 <= 144: the full operators are cheap enough
    if (ctx->m2l_rank > 0) return std::min(ctx->m2l_rank, 4 * n * n) / 8 * 8;
    // 8: 64, 10: 72, 12: 80, 14: 88, 16: 96.  Measured on 20,000 random
    // fracture elements: the product differs from the uncompressed one by
    // about 1e-9 of its block maxima at k = 64 for every n (1e-8 at k = 48),
    // far below the FP32 rounding of the products themselves
    return 64 + 4 * (n - 8);
}

ddm_status svd_build(ddm_ctx *ctx, ddm_tree *t, const float *ops, int k, cudaStream_t s, float *pre, float *post,
                     float *core) {
    const int n = t->prm.n_cheb, n2 = n * n, ld = 4 * n2, L = t->depth;
    if (k <= 0 || k > KMAX) return ctx_fail(ctx, DDM_EINVAL, "compressed M2L: no rank for this order");
    if (t->h_mk_off.empty()) {           // key counts on the host (once per tree)
        t->h_mk_off.resize(t->n_keys + 1);
        DDM_CUDA_TRY(ctx, cudaMemcpyAsync(t->h_mk_off.data(), t->mk_off, (t->n_keys + 1) * sizeof(int32_t),
                                          cudaMemcpyDeviceToHost, s));
        DDM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    // level slots m (levels >= 2 with at least one interaction pair) and
    // their keys (offsets outside the neighbour ring with pairs)
    std::vector<int> lvl, ko{0}, keys;
    for (int l = 2; l <= L; ++l) {
        const size_t before = keys.size();
        for (int o = 0; o < 49; ++o) {
            const int key = l * 49 + o, dx = o / 7 - 3, dy = o % 7 - 3;
            if ((abs(dx) <= 1 && abs(dy) <= 1) || t->h_mk_off[key + 1] == t->h_mk_off[key]) continue;
            keys.push_back(key);
        }
        if (keys.size() == before) continue;
        lvl.push_back(l);
        ko.push_back((int)keys.size());
    }
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(pre, 0, (size_t)(L + 1) * k * ld * sizeof(float), s));
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(post, 0, (size_t)(L + 1) * ld * k * sizeof(float), s));
    DDM_CUDA_TRY(ctx, cudaMemsetAsync(core, 0, (size_t)t->n_keys * k * k * sizeof(float), s));
    const int nl = (int)lvl.size(), nkt = (int)keys.size();
    if (nl == 0) return DDM_OK;
    const int64_t big = (int64_t)ld * ld, kl = (int64_t)k * ld;
    // scratch: T (random test matrices, then core products), P (2 nkt
    // products), Y (2 nl bases), scales, norms
    float *T = nullptr, *P = nullptr, *Y = nullptr, *S = nullptr;
    double *nrm = nullptr;
    int *ibuf = nullptr;
    GDesc *dd = nullptr;
    const int nd = 4 * nkt;                               // range finder (2 nkt); cores (2 sets of nkt)
    const int ni = nkt + (nl + 1) + nl + (2 * nl + 1);    // keys, ko, lvl, zo
    ddm_status st = DDM_OK;
    auto fail = [&](cudaError_t e) {
        return e == cudaSuccess ? DDM_OK : ctx_fail(ctx, DDM_ENOMEM, "compressed M2L: scratch allocation failed");
    };
    if (!st) st = fail(dalloc(&T, (size_t)2 * nkt * kl * sizeof(float), s));
    if (!st) st = fail(dalloc(&P, (size_t)2 * nkt * kl * sizeof(float), s));
    if (!st) st = fail(dalloc(&Y, (size_t)2 * nl * kl * sizeof(float), s));
    if (!st) st = fail(dalloc(&S, (size_t)8 * nl * sizeof(float), s));
    if (!st) st = fail(dalloc(&nrm, (size_t)8 * nl * sizeof(double), s));
    if (!st) st = fail(dalloc(&ibuf, (size_t)ni * sizeof(int), s));
    if (!st) st = fail(dalloc(&dd, (size_t)nd * sizeof(GDesc), s));
    std::vector<GDesc> hd(nd);
    std::vector<int> hi;
    if (!st) {
        // descriptor sets, z = side * nkt + q over (side, level slot, key)
        GDesc *rf = hd.data(), *c1 = rf + 2 * nkt, *c2 = c1 + nkt;
        for (int side = 0; side < 2; ++side)
            for (int m = 0; m < nl; ++m)
                for (int q = ko[m]; q < ko[m + 1]; ++q) {
                    const int z = side * nkt + q;
                    const float *op = ops + (int64_t)keys[q] * big, *so = S + 8 * m, *si = S + 8 * m + 4;
                    // P_z = Omega_z^T op(K~): side 0 (right basis V) Omega^T K~, side 1 (U) Omega^T K~^T
                    rf[z] = GDesc{T + z * kl, op, P + z * kl, so, si, side};
                    if (side == 0) {
                        // cores: T_q = U^T K~ (Ut = Y_{nl + m}), C = T_q V (Vt = Y_m)
                        c1[q] = GDesc{Y + (nl + m) * kl, op, T + q * kl, so, si, 0};
                        c2[q] = GDesc{T + q * kl, Y + m * kl, core + (int64_t)keys[q] * k * k, nullptr, nullptr, 1};
                    }
                }
        hi.insert(hi.end(), keys.begin(), keys.end());
        hi.insert(hi.end(), ko.begin(), ko.end());
        hi.insert(hi.end(), lvl.begin(), lvl.end());
        for (int side = 0; side < 2; ++side)
            for (int m = 0; m < nl; ++m) hi.push_back(side * nkt + ko[m]);
        hi.push_back(2 * nkt);
        if (cudaMemcpyAsync(dd, hd.data(), hd.size() * sizeof(GDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(ibuf, hi.data(), hi.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = ctx_fail(ctx, DDM_ECUDA, "compressed M2L: upload failed");
    }
    if (!st) {
        const int *dkeys = ibuf, *dko = ibuf + nkt, *dlvl = dko + nl + 1, *dzo = dlvl + nl;
        GDesc *rf = dd, *c1 = dd + 2 * nkt, *c2 = dd + 3 * nkt;
        prof_begin(ctx, 3);
        // component equilibration: row scales, then column scales of the row-scaled operators
        cudaMemsetAsync(nrm, 0, (size_t)8 * nl * sizeof(double), s);
        const dim3 ng((unsigned)std::min<int64_t>(1024, (40 * big + 255) / 256), (unsigned)nl);
        k_block_norms<<<ng, 256, 0, s>>>(ops, dkeys, dko, n2, 0, S, nrm);
        k_scales<<<(4 * nl + 127) / 128, 128, 0, s>>>(nrm, nl, 0, S);
        k_block_norms<<<ng, 256, 0, s>>>(ops, dkeys, dko, n2, 1, S, nrm + 4 * nl);
        k_scales<<<(4 * nl + 127) / 128, 128, 0, s>>>(nrm + 4 * nl, nl, 4, S);
        // range finder of both sides on every level: Y = orth(sum_o Omega_o^T op(K~_o))
        k_rand<<<(unsigned)((2 * nkt * kl + 255) / 256), 256, 0, s>>>(T, 2 * nkt * kl, 0x9E3779B9u);
        k_gemm_desc<<<ggrid(k, ld, 2 * nkt), 256, 0, s>>>(k, ld, ld, n2, rf);
        k_sum_parts<<<dim3((unsigned)((kl + 255) / 256), (unsigned)(2 * nl)), 256, 0, s>>>(P, dzo, kl, Y);
        k_orth<<<2 * nl, OT, 0, s>>>(Y, ld, k);
        // cores C_q = U^T K~_q V into their key slots, then the pre- and post-operators
        k_gemm_desc<<<ggrid(k, ld, nkt), 256, 0, s>>>(k, ld, ld, n2, c1);
        k_gemm_desc<<<ggrid(k, k, nkt), 256, 0, s>>>(k, k, ld, n2, c2);
        k_pre_post<<<dim3((unsigned)((kl + 255) / 256), (unsigned)nl), 256, 0, s>>>(Y, nl, S, dlvl, n2, k, pre, post);
        prof_end(ctx, 3, 11);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = ctx_fail(ctx, DDM_ECUDA, cudaGetErrorString(e));
    }
    // the descriptor and index uploads read host vectors that go out of scope
    if (cudaStreamSynchronize(s) != cudaSuccess && !st) st = ctx_fail(ctx, DDM_ECUDA, "compressed M2L: set-up failed");
    void *ps[] = {T, P, Y, S, nrm, ibuf, dd};
    for (void *p : ps) dfree(p, s);
    return st;
}
