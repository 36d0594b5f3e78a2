// Device code of the B300 HPR-LP solver (sm_103a).
//
// The hot path is the HPR iteration of Algorithm 2 with the closed forms of
// Section 3.3 (eq. update-x, update-y-2) and the reflection / Halpern steps:
//
//   phase X (over the rows of A^T, i.e. the columns j of A):
//       s = (A^T y)_j;  v = x_j + sigma (s - c_j);  xbar = Pi_[l_j,u_j](v)
//       xhat_j = 2 xbar - x_j;  x_j <- x0_j/(t+2) + (t+1)/(t+2) xhat_j
//   phase Y (over the rows i of A):
//       q = (A xhat)_i;  ybar = y_i + (b_i - q)/(lambda sigma), clamped at 0 for i >= m1
//       yhat = 2 ybar - y_i;  y_i <- y0_i/(t+2) + (t+1)/(t+2) yhat
//
// Both phases are one CSR SpMV each with the elementwise work fused as an epilogue, so
// every vector crosses HBM once per iteration.  B300 executes FP64 at a small fraction
// of its FP32 rate, so the SpMV spends exactly one FP64 FMA per nonzero: the nonzeros
// of a tile are split evenly over the threads (KPT consecutive nonzeros each), every
// thread accumulates its row fragments with FMA, and fragments of rows that straddle
// threads are combined afterwards in a fixed order.  All reductions (row sums, CTA
// partials, final sums) have a fixed order, so results are bitwise reproducible.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hprdev {

constexpr int TB = 256;                 // threads per tile CTA
constexpr int KPT = 7;                  // nonzeros per thread (odd: conflict-free smem reads)
constexpr int TILE_NNZ = TB * KPT;      // 1792 nonzeros staged per tile
constexpr int TILE_ROWS = TB;           // at most one epilogue row per thread

// quantities reduced at a check (indices into the partials / scalar arrays)
enum {
    Q_DX2 = 0,   // ||x - xbar||^2                      (phase X, check mode)
    Q_XX0 = 1,   // ||xbar - x0||^2
    Q_CX = 2,    // <c_s, xbar>
    Q_BND = 3,   // sum_{z>0} z l_s + sum_{z<0} z u_s
    Q_DY2 = 4,   // ||y - ybar||^2                      (phase Y, check mode)
    Q_YY0 = 5,   // ||ybar - y0||^2
    Q_BY = 6,    // <b_s, ybar>
    Q_RD = 7,    // ||w_c (c_s - A^T ybar - zbar)||^2   (dual residual pass)
    Q_RP = 8,    // ||w_r Pi_D(b_s - A xbar)||^2        (primal residual pass)
    Q_CROSS = 9, // <y - ybar, A (x - xbar)>
    Q_S2 = 10,   // power method: ||A^T u||^2
    Q_W2 = 11,   // power method: ||A A^T u||^2
    Q_V2 = 12,   // generic vector norm (start vector, b, c)
    Q_V2B = 13,
    NQ = 16
};

// Per-period control block written by the host before each check period.
struct DevCtl {
    double sigma;     // sigma_r
    double inv_ls;    // 1 / (lambda sigma_r)
    double pad[6];
    double h[2];      // h[2i] = 1/(t+2), h[2i+1] = (t+1)/(t+2) for iteration i of the period
};

struct PowCtl {
    double lam, lam_prev, inv, tol;
    int k, done, max_iter, stop_after;
};

// ------------------------------------------------------------------ block reduction
// Fixed-order sum of one double per thread over a TB-thread block; result valid in
// thread 0.  Order: xor-butterfly inside each warp, then the 8 warp sums in order.
__device__ __forceinline__ double block_sum(double v, double *scratch /* >= TB/32 */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        s = scratch[0];
#pragma unroll
        for (int i = 1; i < TB / 32; ++i) s += scratch[i];
    }
    return s;
}

// ------------------------------------------------------------------ tile SpMV
template <int NV>
struct TileSmem {
    double val[TILE_NNZ];
    int col[TILE_NNZ];
    int rp[TILE_ROWS + 1];
    double sum[NV][TILE_ROWS];
    double tail[NV][TB];
    double red[TB / 32];
};

// Row sums of rows [r0, r1) of a CSR matrix against NV dense vectors, left in
// sm.sum[v][row - r0].  A tile holds either at most TILE_ROWS rows with at most
// TILE_NNZ nonzeros in total, or a single longer row.
template <int NV>
__device__ __forceinline__ void tile_spmv(const int *__restrict__ rp, const int *__restrict__ ci,
                                          const double *__restrict__ val,
                                          const double *__restrict__ xa,
                                          const double *__restrict__ xb, int r0, int r1,
                                          TileSmem<NV> &sm)
{
    const int tid = threadIdx.x;
    const int R = r1 - r0;
    const int p0 = rp[r0];
    const int N = rp[r1] - p0;

    if (N > TILE_NNZ) {
        // one long row: strided coalesced FMA accumulation, then a fixed-order tree
        double acc0 = 0.0, acc1 = 0.0;
        for (int p = p0 + tid; p < p0 + N; p += TB) {
            const double a = val[p];
            const int c = ci[p];
            acc0 = fma(a, __ldg(xa + c), acc0);
            if (NV == 2) acc1 = fma(a, __ldg(xb + c), acc1);
        }
        double s0 = block_sum(acc0, sm.red);
        if (tid == 0) sm.sum[0][0] = s0;
        if (NV == 2) {
            double s1 = block_sum(acc1, sm.red);
            if (tid == 0) sm.sum[NV - 1][0] = s1;
        }
        __syncthreads();
        return;
    }

    // stage the tile's nonzeros and row pointers (coalesced)
    for (int i = tid; i < N; i += TB) {
        sm.val[i] = val[p0 + i];
        sm.col[i] = ci[p0 + i];
    }
    for (int i = tid; i <= R; i += TB) sm.rp[i] = rp[r0 + i] - p0;
    for (int i = tid; i < R; i += TB) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sm.sum[v][i] = 0.0;
    }
    __syncthreads();

    const int a = tid * KPT;
    int head_row = -1;
    double head[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) head[v] = 0.0;

    if (a < N) {
        const int b = min(a + KPT, N);
        // row holding nonzero a: sm.rp[lo] <= a < sm.rp[lo+1]
        int lo = 0, hi = R;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sm.rp[mid] <= a) lo = mid;
            else hi = mid;
        }
        int row = lo;
        int row_start = sm.rp[row];
        int row_end = sm.rp[row + 1];

        double vv[KPT], g0[KPT], g1[KPT];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int p = a + k;
            if (p < b) {
                const int c = sm.col[p];
                vv[k] = sm.val[p];
                g0[k] = __ldg(xa + c);
                if (NV == 2) g1[k] = __ldg(xb + c);
            }
        }
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0.0;
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int p = a + k;
            if (p < b) {
                while (row_end <= p) {
                    // the current row ends before p: emit its fragment
                    if (row_start < a) {
                        head_row = row;
#pragma unroll
                        for (int v = 0; v < NV; ++v) head[v] = acc[v];
                    } else {
#pragma unroll
                        for (int v = 0; v < NV; ++v) sm.sum[v][row] = acc[v];
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
                    ++row;
                    row_start = row_end;
                    row_end = sm.rp[row + 1];
                }
                acc[0] = fma(vv[k], g0[k], acc[0]);
                if (NV == 2) acc[NV - 1] = fma(vv[k], g1[k], acc[NV - 1]);
            }
        }
        if (row_end == b) {
            if (row_start < a) {
                head_row = row;
#pragma unroll
                for (int v = 0; v < NV; ++v) head[v] = acc[v];
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) sm.sum[v][row] = acc[v];
            }
        } else {
            // the row continues in the next thread(s)
#pragma unroll
            for (int v = 0; v < NV; ++v) sm.tail[v][tid] = acc[v];
        }
    }
    __syncthreads();
    if (head_row >= 0) {
        // this thread holds the last fragment of a row that started in thread t0:
        // sum the fragments in thread order
        const int t0 = sm.rp[head_row] / KPT;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double s = sm.tail[v][t0];
            for (int t = t0 + 1; t < tid; ++t) s += sm.tail[v][t];
            sm.sum[v][head_row] = s + head[v];
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ HPR phase X
struct XArgs {
    const int *tiles, *rp, *ci;   // CSR of A^T (rows = columns of A)
    const double *val;
    const double *y;              // gathered
    const double *c, *l, *u, *x0;
    double *x, *xhat;
    double *xbar, *zbar, *dx;     // check mode only
    double *partials;
    int pstride;
    const DevCtl *ctl;
};

template <bool CHECK>
__global__ void __launch_bounds__(TB) k_phase_x(XArgs A, int it)
{
    __shared__ TileSmem<1> sm;
    const int r0 = A.tiles[blockIdx.x], r1 = A.tiles[blockIdx.x + 1];
    tile_spmv<1>(A.rp, A.ci, A.val, A.y, nullptr, r0, r1, sm);
    const double sigma = A.ctl->sigma;
    const double ha = A.ctl->h[2 * it], hb = A.ctl->h[2 * it + 1];
    double p_dx = 0.0, p_xx0 = 0.0, p_cx = 0.0, p_bnd = 0.0;
    for (int i = threadIdx.x; i < r1 - r0; i += TB) {
        const int j = r0 + i;
        const double xj = A.x[j];
        const double cj = A.c[j], lj = A.l[j], uj = A.u[j], x0j = A.x0[j];
        const double v = fma(sigma, sm.sum[0][i] - cj, xj);   // x + sigma (A^T y - c)
        const double xb = fmin(fmax(v, lj), uj);               // Pi_C, eq. (update-x)
        const double xh = 2.0 * xb - xj;                       // reflection
        A.xhat[j] = xh;
        A.x[j] = fma(hb, xh, ha * x0j);                        // Halpern step
        if (CHECK) {
            const double zb = (xb - v) / sigma;                // eq. (update-z)
            const double d = xj - xb;
            A.xbar[j] = xb;
            A.zbar[j] = zb;
            A.dx[j] = d;
            p_dx = fma(d, d, p_dx);
            p_xx0 = fma(xb - x0j, xb - x0j, p_xx0);
            p_cx = fma(cj, xb, p_cx);
            if (zb > 0.0) p_bnd = fma(zb, lj, p_bnd);
            else if (zb < 0.0) p_bnd = fma(zb, uj, p_bnd);
        }
    }
    if (CHECK) {
        double s;
        s = block_sum(p_dx, sm.red);  if (threadIdx.x == 0) A.partials[Q_DX2 * A.pstride + blockIdx.x] = s;
        s = block_sum(p_xx0, sm.red); if (threadIdx.x == 0) A.partials[Q_XX0 * A.pstride + blockIdx.x] = s;
        s = block_sum(p_cx, sm.red);  if (threadIdx.x == 0) A.partials[Q_CX * A.pstride + blockIdx.x] = s;
        s = block_sum(p_bnd, sm.red); if (threadIdx.x == 0) A.partials[Q_BND * A.pstride + blockIdx.x] = s;
    }
}

// ------------------------------------------------------------------ HPR phase Y
struct YArgs {
    const int *tiles, *rp, *ci;   // CSR of A
    const double *val;
    const double *xhat;           // gathered
    const double *b, *y0;
    double *y;
    double *ybar, *dy;            // check mode only
    double *partials;
    int pstride;
    int m1;
    const DevCtl *ctl;
};

template <bool CHECK>
__global__ void __launch_bounds__(TB) k_phase_y(YArgs A, int it)
{
    __shared__ TileSmem<1> sm;
    const int r0 = A.tiles[blockIdx.x], r1 = A.tiles[blockIdx.x + 1];
    tile_spmv<1>(A.rp, A.ci, A.val, A.xhat, nullptr, r0, r1, sm);
    const double inv_ls = A.ctl->inv_ls;
    const double ha = A.ctl->h[2 * it], hb = A.ctl->h[2 * it + 1];
    double p_dy = 0.0, p_yy0 = 0.0, p_by = 0.0;
    for (int ii = threadIdx.x; ii < r1 - r0; ii += TB) {
        const int i = r0 + ii;
        const double yi = A.y[i], bi = A.b[i], y0i = A.y0[i];
        double yb = fma(bi - sm.sum[0][ii], inv_ls, yi);       // eq. (update-y-2)
        if (i >= A.m1) yb = fmax(yb, 0.0);                     // Pi_{R^m2_+}
        const double yh = 2.0 * yb - yi;                       // reflection
        A.y[i] = fma(hb, yh, ha * y0i);                        // Halpern step
        if (CHECK) {
            const double d = yi - yb;
            A.ybar[i] = yb;
            A.dy[i] = d;
            p_dy = fma(d, d, p_dy);
            p_yy0 = fma(yb - y0i, yb - y0i, p_yy0);
            p_by = fma(bi, yb, p_by);
        }
    }
    if (CHECK) {
        double s;
        s = block_sum(p_dy, sm.red);  if (threadIdx.x == 0) A.partials[Q_DY2 * A.pstride + blockIdx.x] = s;
        s = block_sum(p_yy0, sm.red); if (threadIdx.x == 0) A.partials[Q_YY0 * A.pstride + blockIdx.x] = s;
        s = block_sum(p_by, sm.red);  if (threadIdx.x == 0) A.partials[Q_BY * A.pstride + blockIdx.x] = s;
    }
}

// ------------------------------------------------------------------ check passes
// dual residual (Section 4.1) in original-space weights w_c = beta_c / D_c
struct DualArgs {
    const int *tiles, *rp, *ci;
    const double *val;
    const double *ybar, *c, *zbar, *wc;
    double *partials;
    int pstride;
};

__global__ void __launch_bounds__(TB) k_check_dual(DualArgs A)
{
    __shared__ TileSmem<1> sm;
    const int r0 = A.tiles[blockIdx.x], r1 = A.tiles[blockIdx.x + 1];
    tile_spmv<1>(A.rp, A.ci, A.val, A.ybar, nullptr, r0, r1, sm);
    double p = 0.0;
    for (int i = threadIdx.x; i < r1 - r0; i += TB) {
        const int j = r0 + i;
        const double r = A.wc[j] * (A.c[j] - sm.sum[0][i] - A.zbar[j]);
        p = fma(r, r, p);
    }
    const double s = block_sum(p, sm.red);
    if (threadIdx.x == 0) A.partials[Q_RD * A.pstride + blockIdx.x] = s;
}

// primal residual with weights w_r = beta_b / D_r, and the cross term <dy, A dx> of
// the M-norm (eq. def:M with T1 = lambda I - A A^*)
struct PrimalArgs {
    const int *tiles, *rp, *ci;
    const double *val;
    const double *xbar, *dx, *b, *wr, *dy;
    double *partials;
    int pstride;
    int m1;
};

__global__ void __launch_bounds__(TB) k_check_primal(PrimalArgs A)
{
    __shared__ TileSmem<2> sm;
    const int r0 = A.tiles[blockIdx.x], r1 = A.tiles[blockIdx.x + 1];
    tile_spmv<2>(A.rp, A.ci, A.val, A.xbar, A.dx, r0, r1, sm);
    double pr = 0.0, pc = 0.0;
    for (int ii = threadIdx.x; ii < r1 - r0; ii += TB) {
        const int i = r0 + ii;
        double r = A.b[i] - sm.sum[0][ii];
        if (i >= A.m1) r = fmax(r, 0.0);                       // Pi_D
        r *= A.wr[i];
        pr = fma(r, r, pr);
        pc = fma(A.dy[i], sm.sum[1][ii], pc);
    }
    double s = block_sum(pr, sm.red);
    if (threadIdx.x == 0) A.partials[Q_RP * A.pstride + blockIdx.x] = s;
    s = block_sum(pc, sm.red);
    if (threadIdx.x == 0) A.partials[Q_CROSS * A.pstride + blockIdx.x] = s;
}

// ------------------------------------------------------------------ final reduction
struct RedSpec {
    int nq;
    int q[NQ];
    int cnt[NQ];
};

// out[q] = sum of partials[q][0..cnt) in a fixed order (one CTA per quantity)
__global__ void __launch_bounds__(TB) k_reduce(const double *__restrict__ partials, int pstride,
                                               RedSpec spec, double *out, const int *skip)
{
    __shared__ double red[TB / 32];
    if (skip && *skip) return;
    const int q = spec.q[blockIdx.x], cnt = spec.cnt[blockIdx.x];
    double s = 0.0;
    for (int g = threadIdx.x; g < cnt; g += TB) s += partials[q * pstride + g];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[q] = s;
}

// ------------------------------------------------------------------ restart
// w^{r+1,0} = w_bar (Algorithm 2): x = x0 = xbar, y = y0 = ybar
__global__ void k_restart(int n, int m, const double *__restrict__ xbar,
                          const double *__restrict__ ybar, double *x, double *x0, double *y,
                          double *y0)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            const double v = xbar[i];
            x[i] = v;
            x0[i] = v;
        } else {
            const double v = ybar[i - n];
            y[i - n] = v;
            y0[i - n] = v;
        }
    }
}

// back-map of w_bar to the original LP: x = Pi_C(beta_b D_c xbar), y = beta_c D_r ybar,
// z = beta_c zbar / D_c
__global__ void k_backmap(int n, int m, double beta_b, double beta_c, const double *xbar,
                          const double *ybar, const double *zbar, const double *Dr,
                          const double *Dc, const double *lo, const double *uo, double *xo,
                          double *yo, double *zo)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            xo[i] = fmin(fmax(beta_b * Dc[i] * xbar[i], lo[i]), uo[i]);
            zo[i] = beta_c * zbar[i] / Dc[i];
        } else {
            yo[i - n] = beta_c * Dr[i - n] * ybar[i - n];
        }
    }
}

// ------------------------------------------------------------------ power method
// SplitMix64 (Steele, Lea & Flood 2014): i-th output of the stream started at seed
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// u_i = 2 U_i - 1 and the partial ||u||^2 (one partial per CTA)
__global__ void __launch_bounds__(TB) k_pow_start(int m, uint64_t seed, double *u,
                                                  double *partials, int pstride)
{
    __shared__ double red[TB / 32];
    double p = 0.0;
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i < m) {
        const double v = 2.0 * ((double)(splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
        u[i] = v;
        p = v * v;
    }
    const double s = block_sum(p, red);
    if (threadIdx.x == 0) partials[Q_V2 * pstride + blockIdx.x] = s;
}

struct SpmvNormArgs {
    const int *tiles, *rp, *ci;
    const double *val;
    const double *xin;
    double *out;
    double *partials;
    int pstride, q;
    const PowCtl *pc;   // skip when pc->done (may be NULL)
};

// out = M xin over the tile rows and the partial ||out||^2
__global__ void __launch_bounds__(TB) k_spmv_norm(SpmvNormArgs A)
{
    __shared__ TileSmem<1> sm;
    if (A.pc && A.pc->done) return;
    const int r0 = A.tiles[blockIdx.x], r1 = A.tiles[blockIdx.x + 1];
    tile_spmv<1>(A.rp, A.ci, A.val, A.xin, nullptr, r0, r1, sm);
    double p = 0.0;
    for (int i = threadIdx.x; i < r1 - r0; i += TB) {
        const double v = sm.sum[0][i];
        A.out[r0 + i] = v;
        p = fma(v, v, p);
    }
    const double s = block_sum(p, sm.red);
    if (threadIdx.x == 0) A.partials[A.q * A.pstride + blockIdx.x] = s;
}

// after s = A^T u: lambda_k = ||s||^2; stop when |lambda_k - lambda_{k-1}| <= tol lambda_k
__global__ void k_pow_after_s(PowCtl *pc, const double *scal)
{
    if (pc->done) return;
    pc->k += 1;
    pc->lam = scal[Q_S2];
    if (pc->k > 1 && fabs(pc->lam - pc->lam_prev) <= pc->tol * pc->lam) {
        pc->done = 1;
        return;
    }
    pc->lam_prev = pc->lam;
    if (pc->k >= pc->max_iter) pc->stop_after = 1;
}

// after w = A s: 1 / ||w|| for the normalisation
__global__ void k_pow_after_w(PowCtl *pc, const double *scal)
{
    if (pc->done) return;
    const double nw = sqrt(scal[Q_W2]);
    if (!(nw > 0.0)) {
        pc->done = 1;
        return;
    }
    pc->inv = 1.0 / nw;
}

__global__ void k_pow_finish(PowCtl *pc)
{
    if (!pc->done && pc->stop_after) pc->done = 1;
}

// u = w * inv (skipped once done)
__global__ void k_scale_vec(int m, const double *w, double *u, const PowCtl *pc, const double *inv_ptr)
{
    if (pc && pc->done) return;
    const double inv = inv_ptr ? *inv_ptr : pc->inv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        u[i] = w[i] * inv;
}

__global__ void k_inv_sqrt_scalar(const double *scal, int q, double *out)
{
    *out = 1.0 / sqrt(scal[q]);
}

// ------------------------------------------------------------------ preprocessing
__global__ void k_gather(int64_t nnz, const double *__restrict__ src, const int *__restrict__ perm,
                         double *dst)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[perm[k]];
}

// d_i = max_p |val_p| over row i, in index order
__global__ void k_row_absmax(int rows, const int *__restrict__ rp, const double *__restrict__ val,
                             double *d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        double mx = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const double a = fabs(val[p]);
            if (a > mx) mx = a;
        }
        d[i] = mx;
    }
}

// d_i = sum_p |val_p|^e over row i, in index order (e == 1: plain |val|)
__global__ void k_row_abspow(int rows, const int *__restrict__ rp, const double *__restrict__ val,
                             double e, double *d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const double a = fabs(val[p]);
            s += (e == 1.0) ? a : pow(a, e);
        }
        d[i] = s;
    }
}

// d = d > 0 ? 1/sqrt(d) : 1;  D *= d
__global__ void k_factor(int rows, double *d, double *D)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const double v = d[i] > 0.0 ? 1.0 / sqrt(d[i]) : 1.0;
        d[i] = v;
        D[i] *= v;
    }
}

// a_ij <- a_ij * dr_i * dc_j
__global__ void k_scale_rows_cols(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                                  double *val, const double *__restrict__ dr,
                                  const double *__restrict__ dc)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const double r = dr[i];
        for (int p = rp[i]; p < rp[i + 1]; ++p) val[p] = val[p] * r * dc[ci[p]];
    }
}

// b~ = D_r b, c~ = D_c c, l~ = l / D_c, u~ = u / D_c, and the partials of ||b~||^2,
// ||c~||^2 (grid over max(m, n) entries, one partial per CTA)
__global__ void __launch_bounds__(TB) k_prep_vectors(int m, int n, const double *Dr,
                                                     const double *Dc, double *b, double *c,
                                                     double *l, double *u, double *partials,
                                                     int pstride)
{
    __shared__ double red[TB / 32];
    const int i = blockIdx.x * TB + threadIdx.x;
    double pb = 0.0, pcn = 0.0;
    if (i < m) {
        const double v = b[i] * Dr[i];
        b[i] = v;
        pb = v * v;
    }
    if (i < n) {
        const double v = c[i] * Dc[i];
        c[i] = v;
        pcn = v * v;
        l[i] = l[i] / Dc[i];
        u[i] = u[i] / Dc[i];
    }
    double s = block_sum(pb, red);
    if (threadIdx.x == 0) partials[Q_V2 * pstride + blockIdx.x] = s;
    s = block_sum(pcn, red);
    if (threadIdx.x == 0) partials[Q_V2B * pstride + blockIdx.x] = s;
}

// b_s = b~ / beta_b, l_s, u_s likewise, c_s = c~ / beta_c; weights of the residuals in
// the original space w_r = beta_b / D_r, w_c = beta_c / D_c
__global__ void k_prep_normalise(int m, int n, double beta_b, double beta_c, const double *Dr,
                                 const double *Dc, double *b, double *c, double *l, double *u,
                                 double *wr, double *wc)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (m > n ? m : n);
         i += gridDim.x * blockDim.x) {
        if (i < m) {
            b[i] = b[i] / beta_b;
            wr[i] = beta_b / Dr[i];
        }
        if (i < n) {
            c[i] = c[i] / beta_c;
            l[i] = l[i] / beta_b;
            u[i] = u[i] / beta_b;
            wc[i] = beta_c / Dc[i];
        }
    }
}

__global__ void k_fill(int64_t n, double v, double *d)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = v;
}

}  // namespace hprdev
