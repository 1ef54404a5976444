// Fracture growth step (paper Sec. 4: the time-marching algorithm checks the
// propagation of every tip after a step's solve and adds tip elements; the
// paper gives no criterion, the reading below supplies the standard one).
//
// Per tip element (its half-length a, the tip at its end `end`): K_I, K_II
// by Olson's tip formula (Eq. 2.6, as ddm_sif), expressed in the crack-tip
// frame (x outward along the fracture, y = x turned by +90 degrees; with the
// opening Dn > 0 both ends see the same signs as the element frame).  The
// maximum tangential stress criterion (Erdogan and Sih) gives the kink angle
//     theta = 2 atan((K_I - sqrt(K_I^2 + 8 K_II^2)) / (4 K_II))   (0 if K_II = 0)
// and the equivalent mode-I factor
//     K_eq = cos(theta/2) (K_I cos^2(theta/2) - 1.5 K_II sin(theta)).
// A tip with K_I > 0 and K_eq >= K_Ic grows by one element of the tip
// element's length along x rotated by theta; the new element runs from the
// old tip point to the new one, so its end 1 is the new tip.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

// per tip: theta, K_eq, growth flag and the new segment (x0, y0, x1, y1)
__global__ void k_grow_eval(const double *xy, int64_t n, const double *x, const int64_t *tip, const int *end, int m,
                            double G, double nu, double KIc, double *theta, double *keq, int *flag, double *seg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t e = tip[i];
    const double ax = xy[e], ay = xy[n + e], bx = xy[2 * n + e], by = xy[3 * n + e];
    const double L = hypot(bx - ax, by - ay), a = 0.5 * L;
    const double E = 2.0 * G * (1.0 + nu);
    const double f = 0.806 * E / (4.0 * (1.0 - nu * nu)) * sqrt(M_PI / (2.0 * a));
    const double KI = f * x[n + e], KII = f * x[e];
    const double th = KII != 0.0 ? 2.0 * atan((KI - sqrt(KI * KI + 8.0 * KII * KII)) / (4.0 * KII)) : 0.0;
    const double c = cos(0.5 * th);
    const double K = c * (KI * c * c - 1.5 * KII * sin(th));
    // crack-tip frame: x outward along the element, y = x turned by +90 degrees
    const double sx = end[i] ? 1.0 : -1.0;
    const double txx = sx * (bx - ax) / L, txy = sx * (by - ay) / L;
    const double tyx = -txy, tyy = txx;
    const double px = end[i] ? bx : ax, py = end[i] ? by : ay;
    const double dx = cos(th) * txx + sin(th) * tyx, dy = cos(th) * txy + sin(th) * tyy;
    theta[i] = th;
    keq[i] = K;
    flag[i] = (KI > 0.0 && K >= KIc) ? 1 : 0;
    seg[4 * i] = px;
    seg[4 * i + 1] = py;
    seg[4 * i + 2] = px + L * dx;
    seg[4 * i + 3] = py + L * dy;
}

// the grown geometry: the n old elements then the new ones, rows of stride n2
__global__ void k_grow_write(const double *xy, int64_t n, const double *seg, const int *flag, const int *slot, int m,
                             int64_t n2, double *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        for (int r = 0; r < 4; ++r) out[r * n2 + i] = xy[r * n + i];
    } else if (i < n + m) {
        const int t = (int)(i - n);
        if (!flag[t]) return;
        const int64_t j = n + slot[t];
        for (int r = 0; r < 4; ++r) out[r * n2 + j] = seg[4 * t + r];
    }
}

// grown tips become the new elements, tip at their end 1
__global__ void k_grow_tips(const int *flag, const int *slot, int m, int64_t n, int64_t *tip, int *end) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !flag[i]) return;
    tip[i] = n + slot[i];
    end[i] = 1;
}

}  // namespace

extern "C" ddm_status ddm_grow(ddm_ctx *ctx, const double *d_xy, int64_t n, const double *d_x, int64_t *d_tip,
                               int *d_tip_end, int n_tips, double K_Ic, double *d_xy_out, int64_t *n_out,
                               double *d_theta, double *d_keq) {
    if (!ctx || !d_xy || n <= 0 || !d_x || n_tips < 0 || (n_tips > 0 && (!d_tip || !d_tip_end)) || !d_xy_out ||
        !n_out || !(K_Ic >= 0.0))
        return ctx_fail(ctx, DDM_EINVAL, "ddm_grow: bad arguments");
    cudaStream_t s = ctx->stream;
    const int m = n_tips;
    double *theta = d_theta, *keq = d_keq, *seg = nullptr;
    int *flag = nullptr, *slot = nullptr;
    double *own = nullptr;                    // theta / K_eq when the caller wants neither
    ddm_status st = DDM_OK;
    const size_t mm = (size_t)std::max(m, 1);
    if (dalloc(&seg, 4 * mm * sizeof(double), s) != cudaSuccess || dalloc(&flag, mm * sizeof(int), s) != cudaSuccess ||
        dalloc(&slot, mm * sizeof(int), s) != cudaSuccess || dalloc(&own, 2 * mm * sizeof(double), s) != cudaSuccess)
        st = ctx_fail(ctx, DDM_ENOMEM, "ddm_grow: workspace");
    if (!theta) theta = own;
    if (!keq) keq = own + mm;
    std::vector<int> hf(mm, 0), hs(mm, 0);
    int grown = 0;
    if (!st && m > 0) {
        k_grow_eval<<<(m + 127) / 128, 128, 0, s>>>(d_xy, n, d_x, d_tip, d_tip_end, m, ctx->mat.G, ctx->mat.nu, K_Ic,
                                                    theta, keq, flag, seg);
        if (cudaMemcpyAsync(hf.data(), flag, m * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = ctx_fail(ctx, DDM_ECUDA, "ddm_grow: evaluation failed");
        for (int i = 0; i < m && !st; ++i) {
            hs[i] = grown;
            grown += hf[i];
        }
        if (!st && cudaMemcpyAsync(slot, hs.data(), m * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = ctx_fail(ctx, DDM_ECUDA, "ddm_grow: upload failed");
    }
    const int64_t n2 = n + grown;
    if (!st) {
        k_grow_write<<<(unsigned)((n + m + 255) / 256), 256, 0, s>>>(d_xy, n, seg, flag, slot, m, n2, d_xy_out);
        if (m > 0) k_grow_tips<<<(m + 127) / 128, 128, 0, s>>>(flag, slot, m, n, d_tip, d_tip_end);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = ctx_fail(ctx, DDM_ECUDA, cudaGetErrorString(e));
    }
    // the slot upload reads a host vector: done before it goes out of scope
    if (cudaStreamSynchronize(s) != cudaSuccess && !st) st = ctx_fail(ctx, DDM_ECUDA, "ddm_grow failed");
    dfree(seg, s);
    dfree(flag, s);
    dfree(slot, s);
    dfree(own, s);
    if (!st) *n_out = n2;
    return st;
}
