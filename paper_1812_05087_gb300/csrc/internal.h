// Internal structures shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/ddm.h"

#define DDM_MAX_CHEB 16
#define DDM_MAX_LEVELS 18

// Kernel constants derived from the material (Biot / Rice-Cleary plane
// strain), in the precision T of the arithmetic that uses them.
template <class T>
struct KConst {
    T G2;      // 2G
    T Cel;     // G / (2 pi (1 - nu))           drained elastic DD prefactor
    T Ce;      // (1 - 2 nu) / (2 pi (1 - nu))   drained dilatation prefactor
    T K2;      // kpsi * Ce / 4                   displacement-potential prefactor
    T aS;      // alpha / S                        undrained pore-pressure coefficient
    T eta;     // poroelastic stress coefficient alpha (1 - 2nu) / (2 (1 - nu))
    T i4pk;    // 1 / (4 pi kappa)                 line-source pressure prefactor
    T c;       // hydraulic diffusivity kappa / S
    // products of the above used by the large-u point kernel
    T Cu;      // Cel + 2 G2 K2                    undrained elastic prefactor
    T pS;      // aS Ce                            undrained pressure prefactor
    T a6;      // 6 G2 K2                          linear-in-time stress term
    T qe;      // eta / (4 pi kappa)               linear-in-time fluid-source stress term
};

// Time window of one product: [K(tau_hi) - K(tau_lo)], K(0) = 0.
// ct_* = c * tau_*; elastic = 1 when tau_lo == 0 (the drained elastic part
// cancels between two positive times).
template <class T>
struct Win {
    T ct_hi, ct_lo;
    T g_hi, g_lo;      // 1/(4 ct_*) (0 when ct_* = 0)
    int elastic;
    T rbig;            // distance beyond which u > Big on both sides: sqrt(Big / g_hi)
};

struct ddm_tree {
    cudaStream_t stream;       // stream of the build; frees are ordered on it
    ddm_fmm_params prm;        // FMM parameters of this tree (order, leaf size, depth cap, near rule)
    int64_t n;                 // elements
    int depth;                 // deepest level (the leaf level of a uniform tree)
    int adaptive;              // leaves at any level (cells of > leaf_size elements split)
    double cx, cy, h0;         // root square centre and half-width
    // per level l = 0..L: non-empty cells [lvl_off[l], lvl_off[l+1])
    std::vector<int64_t> lvl_off;
    int64_t n_cells;
    // device arrays
    int64_t *perm;             // sorted position -> caller element index
    uint32_t *cell_key;        // Morton key of each cell at its level (cells sorted by level, key)
    int32_t *cell_ix, *cell_iy;// integer cell coordinates at the cell's level
    int32_t *cell_start, *cell_end;   // sorted element range
    int32_t *cell_parent;      // global cell index of the parent (-1 at level 0)
    int32_t *il_off, *il_idx;  // interaction lists (CSR over cells)
    // leaves: (global cell index, level) of each, in cell order
    int2 *leaf_at = nullptr;
    int64_t n_leaf = 0;
    int leaf_level_min = 0;
    // direct-interaction records of every leaf (CSR over leaves): the element
    // ranges it interacts with directly, (element start, count, 0, 0)
    int32_t *nb_off = nullptr;
    int4 *nb_tab = nullptr;
    int max_recs = 0;          // most records of one leaf
    int2 *near_items;          // near-field work items: target pairs of one leaf (second -1: single)
    int64_t n_items;
    int4 *up_items = nullptr;  // upward-pass work items: (leaf, first element, end, 0)
    int64_t n_up_items = 0;
    int32_t *elem_leaf;        // sorted element -> leaf index (leaf-local)
    // sorted element geometry, FP32 relative to the element's leaf centre
    float4 *g_rel;             // (x0, y0, x1, y1) rel. to leaf centre (expansions)
    float4 *g_frame;           // (tx, ty, half-length, 0)
    // pair geometry of the near field and the dense product: the element's
    // grid point (midpoint cell of the 2^16 x 2^16 key grid, index as exact
    // floats) and its end points relative to that point, so that the
    // displacement of two elements is (g_s - g_t) g16 + (loc_s - loc_t),
    // exact to FP32 rounding of the displacement itself
    float2 *g_grid = nullptr;
    float4 *g_loc = nullptr;
    float g16 = 0.f;
    double *xy_sorted;         // 4 x n FP64 absolute end points (sorted order)
    double *xy_caller;         // 4 x n FP64 end points, caller order (copy of the input)
    // Per time window (tau_lo, tau_hi) caches, least recently used first out:
    // own-element 3x3 blocks and M2L operator sets.  A time-marching run sees
    // the same lag windows every step, and the history sum one per lag.
    static constexpr int WIN_CACHE = 128;
    double *win_blk[WIN_CACHE] = {};
    double win_lo[WIN_CACHE], win_hi[WIN_CACHE];
    unsigned long long win_use[WIN_CACHE] = {};
    int64_t n_m2l, n_p2p;
    // preconditioner blocks: runs of <= 64 elements along chains of elements
    // that share end points (one fracture), caller element indices
    int64_t n_pblk;
    int32_t *pb_off;           // CSR over blocks (elements)
    int64_t *pb_elem;          // caller element index, chain order
    int64_t *pb_moff;          // offset of each block's (3m x 3m) matrix
    int64_t pb_msize;          // total matrix entries
    int pb_max;                // largest block (elements)
    float *pb_inv;             // inverted system blocks of the cached (dt, system), FP32
    double pb_dt;
    int pb_sys;
    // coarse level of the preconditioner: the blocks of long chains (at least
    // PC_MIN_BLOCKS blocks), pc_modes Legendre modes per block and unknown
    // component; pc_inv = inverse of the Galerkin coarse matrix Z^T A Z of the
    // cached (dt, system), FP32, dimension n_pc * nc * pc_modes
    int64_t n_pc;
    int pc_modes;
    int32_t *pc_blk;           // block index of every coarse block
    float *pc_inv;
    bool pc_pending = false;   // coarse matrix assembled, not yet inverted
    // M2L pairs grouped by (level, cell offset): key = level * 49 + (dx+3)*7 + (dy+3)
    int n_keys;                // (L + 1) * 49
    int32_t *mk_off;           // CSR over keys
    int2 *mk_pair;             // (target cell, source cell), global cell indices
    int max_group;             // largest (level, offset) group
    int2 *mk_work;             // (key, first pair) of every 64-pair column tile
    int n_work;
    // M2L operators of the current time window, one (4n^2 x 4n^2) matrix per key
    float *ops_set[WIN_CACHE] = {};
    double ops_lo[WIN_CACHE], ops_hi[WIN_CACHE];
    unsigned long long ops_use[WIN_CACHE] = {};
    unsigned ops_cnt[WIN_CACHE] = {};  // products served by each set (compression policy)
    int ops_n;                 // n_cheb of the cached operator sets
    int ops_cap;               // sets allowed by the memory budget
    unsigned long long win_clock;
    // compressed M2L (svd.cu) of the cached windows: per level a pre-operator
    // (k x 4n^2) and a post-operator (4n^2 x k), per (level, offset) key a
    // k x k core, in one allocation per window
    float *svd_set[WIN_CACHE] = {};
    double svd_lo[WIN_CACHE], svd_hi[WIN_CACHE];
    unsigned long long svd_use[WIN_CACHE] = {};
    std::vector<int32_t> h_mk_off;     // host copy of mk_off (key counts)
    // cells of levels >= 2 as (cell, cell) pairs grouped by level (key =
    // level) with 64-cell work items: the pre- and post-stages
    int32_t *lv_off = nullptr;
    int2 *lv_pair = nullptr, *lv_work = nullptr;
    int n_lv_work = 0;
    float *Wc = nullptr, *Gc = nullptr;  // compressed weights / local sums, k per cell
    int svd_k = 0;                       // rank of the cached compressed sets and of Wc, Gc
    // per-tree workspaces
    float *W;                  // multipole weights, 4 n^2 per cell
    float *Fl;                 // local expansions, 4 n^2 per cell
    float4 *far4;              // far field (global sxx, syy, sxy, p) at each sorted target
    float4 *chg;               // sorted charges (Dx, Dy, q, 0) per element
    int ncheb_alloc;
};

// coarse level of the preconditioner (precond.cu): chains of at least
// PC_MIN_BLOCKS blocks (long fractures, where block Jacobi leaves the
// long-wavelength modes to the Krylov iteration) take PC_MODES modes per
// block, fewer when the coarse dimension would exceed PC_MAX_DIM (its
// set-up is O(dim^3)), none below one mode
constexpr int PC_MIN_BLOCKS = 4, PC_MODES = 3, PC_MAX_DIM = 2048;

struct GmresWork;

// Device state of the GMRES least squares (krylov.cu), P problems of
// restart m: rotated Hessenberg columns H (row-major (m + 1) x m each),
// Givens cosines and sines, the rotated right-hand side g, the solution y of
// R y = g (m + 2 per problem, zero past the cycle's columns), the inner
// targets, the residual estimates |g_{j+1}|, the live flags, the cycle's
// column counts, the iteration counts, the number of problems still live
// after a step, and a status triple of problem 0 (live, |g_{j+1}|, the
// context's error word) for the single solve's per-step read.
struct LsqDev {
    int P = 0, m = 0;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *inner = nullptr, *res = nullptr, *stat = nullptr, *hbuf_dev = nullptr;
    int *live = nullptr, *jend = nullptr, *iters = nullptr, *still = nullptr;
    double *hbuf = nullptr;    // pinned staging of (beta, inner, live0) per problem
    double *hstat = nullptr;   // pinned: two slots of the status triple (plus padding)
    int *hint = nullptr;       // pinned: the still-live count, then P iteration counts
};
ddm_status lsq_alloc(ddm_ctx *ctx, LsqDev &L, int P, int m, cudaStream_t s);
void lsq_free(LsqDev &L, cudaStream_t s);
ddm_status lsq_reset_iters(ddm_ctx *ctx, LsqDev &L, cudaStream_t s);
// start a cycle from host values beta, inner (P each) and live0 (P, or NULL = all)
ddm_status lsq_begin(ddm_ctx *ctx, LsqDev &L, int P, const double *beta, const double *inner, const int *live0,
                     cudaStream_t s);
// Givens step on column j (hcol[p * hstride + i], i <= j + 1) of every live problem
ddm_status lsq_step(ddm_ctx *ctx, LsqDev &L, int P, const double *hcol, int hstride, int j, int max_iters,
                    bool count_still, bool write_stat, cudaStream_t s);
// y = R^{-1} g per problem
ddm_status lsq_solve(ddm_ctx *ctx, LsqDev &L, int P, cudaStream_t s);

// Optional stage timing (CUDA events on the context stream) and launch
// counting.  Stages: 0 prep (charges + own elements), 1 own-element blocks,
// 2 up (fused with prep, P2M, M2M), 3 M2L operators, 4 m2l, 5 down, 6 leaf,
// 7 dense, 8 krylov vector kernels, 9 tree build.
#define DDM_NSTAGES 10
struct Prof {
    int on = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    long long launches[DDM_NSTAGES] = {0};
    int open_stage = -1;
    cudaEvent_t open_ev = nullptr;
};

struct ddm_ctx {
    int device;
    cudaStream_t stream;
    cudaStream_t aux = nullptr;   // far field of a product, concurrent with the near field
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ddm_material mat;
    ddm_fmm_params prm;
    KConst<float> kf;
    KConst<double> kd;
    std::string err;
    // M2M / L2L transfer matrices T[q][a][a'] (device) of every even order n
    // (index n / 2 - 1)
    float *cheb_Tn[DDM_MAX_CHEB / 2] = {};
    GmresWork *gm;
    Prof prof;
    int *d_err;                // device word raised by a kernel whose bounded wait expired
    long long grid_polls = 1ll << 22;   // poll limit of the GMRES grid barriers (ddm_set_wait_limit)
    int m2l_compress = 2;      // compressed M2L: 0 never, 1 always, 2 automatic (ddm_set_m2l_compression)
    int m2l_rank = 0;          // its rank (0: the default per order)
    // time-compressed history (history.cu, ddm_set_history_compression):
    // exact most recent steps (0 = off), nodes per block, block ratio; moment
    // and weight workspaces
    int hist_E = 0, hist_p = 10;
    double hist_rho = 2.0;
    double *hist_M = nullptr, *hist_C = nullptr;
    int64_t hist_M_cap = 0, hist_C_cap = 0;
    double *h_pin = nullptr;   // pinned host staging (tree build: element end points)
    int64_t h_pin_cap = 0;
};

// begin/end a profiled stage (no-ops unless profiling is on); count launches
// Escalated GMRES residuals (precision level >= 1) of problems up to this many
// elements use the exact FP64 dense product (DDM_MODE_DENSE | DDM_MODE_PRECISE),
// once per restart: O(N^2) FP64 pair integrals, about 0.2 s at this size on
// GB300 (FP64 runs at 1/64 of the FP32 rate), which bounds the cost of an
// escalated restart.  Larger problems keep the precise FMM product.
constexpr int64_t EXACT_RES_MAX = 16384;
// largest problem whose escalated Arnoldi products take the exact FP64
// dense product (one per Arnoldi step instead of one per restart)
constexpr int64_t EXACT_OP_MAX = 10000;
inline int residual_mode(int mode, int level, int64_t n) {
    if (level < 1) return mode;
    return (n <= EXACT_RES_MAX ? DDM_MODE_DENSE : (mode & ~DDM_MODE_PRECISE)) | DDM_MODE_PRECISE;
}
// Arnoldi products at an escalation level: the requested ones at levels 0
// and 1, with FP64 direct pairs at level 2, and at level 3 (problems of at
// most EXACT_OP_MAX elements) the exact FP64 dense product, the operator
// their residuals already use from level 1 on
inline int arnoldi_mode(int mode, int level, int64_t n) {
    if (level < 2) return mode;
    if (level >= 3 && n <= EXACT_OP_MAX) return DDM_MODE_DENSE | DDM_MODE_PRECISE;
    return mode | DDM_MODE_PRECISE;
}
inline int max_level(int64_t n) { return n <= EXACT_OP_MAX ? 3 : 2; }

void prof_begin(ddm_ctx *ctx, int stage);
void prof_end(ddm_ctx *ctx, int stage, int launches);

// Device memory comes from the stream-ordered allocator (the device's
// default pool, kept by the process after frees), so that tree builds,
// workspaces and per-request buffers do not synchronise the device.
inline cudaError_t dalloc(void **p, size_t bytes, cudaStream_t s) { return cudaMallocAsync(p, bytes ? bytes : 1, s); }
template <class T> inline cudaError_t dalloc(T **p, size_t bytes, cudaStream_t s) { return dalloc((void **)p, bytes, s); }
inline void dfree(void *p, cudaStream_t s) { if (p) cudaFreeAsync(p, s); }

// error helpers
ddm_status ctx_fail(ddm_ctx *ctx, ddm_status st, const std::string &msg);
#define DDM_CUDA_TRY(ctx, call)                                                        \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess)                                                         \
            return ctx_fail(ctx, DDM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// tree.cu (prm: the tree's FMM parameters, validated by the caller)
ddm_status tree_build(ddm_ctx *ctx, const double *d_xy, int64_t n, const ddm_fmm_params &prm, ddm_tree **out);
void tree_free(ddm_tree *t);

// fmm.cu: y = [K(hi) - K(lo)] x  (caller order), accumulate: y += s * (...)
ddm_status op_apply(ddm_ctx *ctx, ddm_tree *t, double tau_lo, double tau_hi, const double *d_x,
                    double *d_y, int mode, int accumulate, double scale, cudaStream_t stream = nullptr);
// own-element 3x3 blocks (caller order) of window (lo, hi), from the tree's window cache
ddm_status window_self_blocks(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s, const double **out);
ddm_status ensure_workspace(ddm_ctx *ctx, ddm_tree *t);
// M2L operator set of window (lo, hi) for tree t (cached per window)
ddm_status window_ops(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s, const float **out);
// compressed M2L (svd.cu): rank per order (0 = no compression), and the
// bases and cores of one window from its full operators
int svd_rank(const ddm_ctx *ctx, int n);
// products a window's full operators serve before the automatic mode compresses them
constexpr unsigned SVD_AUTO_USES = 128;
bool want_svd(ddm_ctx *ctx, ddm_tree *t, double lo, double hi, cudaStream_t s);
// history sum with the older steps interpolated in log time (history.cu)
ddm_status history_compressed(ddm_ctx *ctx, ddm_tree *t, const double *d_hist, const double *h_times, int H,
                              double *d_rhs, int mode);
ddm_status svd_build(ddm_ctx *ctx, ddm_tree *t, const float *ops, int k, cudaStream_t s, float *pre, float *post,
                     float *core);
// many problems' FMM products, one launch per stage (trees of one order):
// y_p = [K(hi) - K(lo)] x_p for every problem p (fmm.cu)
struct BatchFmm;
// act (device, may be null): per-problem flags read at launch time; problems
// whose flag is 0 are skipped
// trees, xs, ys: all np problems; idx: the nidx members of this work list
// (one order); the descriptor table and act are indexed by problem
ddm_status bfmm_build(ddm_ctx *ctx, ddm_tree *const *trees, int np, const int *idx, int nidx, double lo, double hi,
                      const double *const *xs, double *const *ys, const int *act, cudaStream_t s, BatchFmm **out);
ddm_status bfmm_launch(ddm_ctx *ctx, BatchFmm *b, cudaStream_t s, cudaStream_t aux);
void bfmm_free(BatchFmm *b, cudaStream_t s);
ddm_status upload_tables(ddm_ctx *ctx);
// precond.cu: chain-block Jacobi preconditioner (cached per dt and system)
ddm_status pb_prepare(ddm_ctx *ctx, ddm_tree *t, double dt, int sys, cudaStream_t s, bool defer_coarse = false);
// invert the pending coarse matrices of many trees together
ddm_status pc_invert_many(ddm_ctx *ctx, ddm_tree *const *trees, int count, cudaStream_t s);
ddm_status pb_apply(ddm_ctx *ctx, ddm_tree *t, int sys, const double *v, double *z3, cudaStream_t s);
// the same for many problems in one launch per stage (precond.cu)
struct BatchPb;
ddm_status bpb_build(ddm_ctx *ctx, ddm_tree *const *trees, int np, int sys, const double *const *vs,
                     double *const *zs, const int *act, cudaStream_t s, BatchPb **out);
ddm_status bpb_launch(ddm_ctx *ctx, BatchPb *b, cudaStream_t s);
void bpb_free(BatchPb *b, cudaStream_t s);
