// Persistent grid solve for mid-size LPs: one cooperative launch of G co-resident CTAs runs
// the power method and the whole of Algorithm 2 -- iterations, checks every check_every
// iterations, the restart criteria of Section 3.1, SigmaUpdate (Algorithm 3) and the
// termination test of Section 4.1 -- without returning to the host.
//
// Algorithm 2 has two grid-wide dependencies per iteration: the y step (eq. update-y-2)
// gathers all of x_hat = 2 x_bar - x, and the next x step (eq. update-x) gathers all of y.
// Between kernel launches the stream provides them; here a software grid barrier does (a
// monotonic arrival counter in device memory).  LPs too large for one SM but
// too small to fill the GPU spend most of a launched iteration in launch latency; two
// barriers cost less.
//
// Every barrier wait is bounded: past its time budget a CTA raises the error word and
// returns, every CTA that sees the word returns too, and the host reports
// HPR_ERR_DEVICE_TIMEOUT.  (A cooperative launch guarantees that all G CTAs are resident,
// so a healthy run never waits long.)
//
// Work split: warp g of the grid takes slices g, g + G*NW, ... of the same sliced-ELL
// layouts the multi-CTA path uses, for the whole solve, with the warps numbered CTA-minor
// (g = warp * G + CTA for A, g = warp * G + (CTA + G/2) mod G for A^T): consecutive slices
// go to different CTAs, so the longest slices (rows are numbered by decreasing length)
// spread over all CTAs instead of all landing in the first one.  Every vector that
// this launch writes is written and read through L2 (st/ld.global.cg), never through a
// possibly stale L1 line of another SM; the matrices and the LP data are read-only.
//
// Reductions: each CTA sums its warps' partial sums in a fixed order and publishes them;
// after a barrier EVERY CTA adds the G CTA sums in the same fixed order, so all CTAs hold
// bitwise the same check quantities and take the same decisions (thread 0 of each CTA),
// without a second barrier.  CTA 0 alone writes the check records.
//
// A restart needs no copy pass: in the first iteration of the new inner loop the x step
// reads its own rows' x and x0 from x_bar and gathers y from y_bar, the y step reads its
// own y, y0 from y_bar, and both write the new anchors x0, y0 as they go.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hprgrid {

constexpr int NT = 512;
constexpr int NW = NT / 32;
constexpr int NQG = 10;                      // check quantities (as the single-CTA path's q[])

// barrier state in device memory (zeroed by the host before every launch)
struct GridBar {
    unsigned long long count;                // arrivals so far: barrier nb completes at (nb+1) G
    int err;                                 // 1: a wait ran out of budget
    int where;                               // the barrier number at which it did
};

struct GridArgs {
    int m, n, G;
    hprsmall::SmallMat A, T;                 // A (m rows) and A^T (n rows), renumbered layouts
    const unsigned char *ineq;
    const double *b, *c, *l, *u, *wr, *wc;
    double beta_b, beta_c, norm_b, norm_c;
    double tol, alpha1, alpha2, alpha3, sigma0, lambda_fixed, power_tol;
    int64_t max_iter, check_every, power_max_iter;
    uint64_t seed;
    int restart, sigma_update, halpern, reflect;
    const int *perm_r;
    double *x, *x0, *xh, *xb, *zb, *dx, *y, *y0, *yb, *dy;   // iterates (renumbered)
    double *partials;                        // NQG * G CTA sums
    GridBar *bar;
    uint64_t budget_ns;                      // longest wait at a barrier
    int skip_cta, skip_at;                   // fault injection: CTA skip_cta does not arrive
                                             // at barrier number skip_at (-1: off)
    hpr_check_record *recs;
    int rec_cap;
    double *out;                             // hprsmall::SO_LEN values
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void add_release(unsigned long long *p)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

// Grid-wide barrier number `nb` (every CTA calls the barriers in the same order, once each):
// thread 0 adds its arrival to a monotonic counter with release semantics and polls it with
// acquire loads until all G CTAs have arrived at this barrier, (nb+1) G arrivals in all; the
// CTA barriers before and after pass the order on to the other threads.  Every 64 polls it
// checks the error word and its time budget.  Returns false on every thread of the CTA if a
// wait of the launch ran out of budget: the caller then returns.
__device__ __forceinline__ bool grid_sync(const GridArgs &P, int nb, int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        GridBar *B = P.bar;
        int ok = 1;
        const unsigned long long target = (unsigned long long)(nb + 1) * (unsigned long long)P.G;
        if (!(blockIdx.x == (unsigned)P.skip_cta && nb == P.skip_at)) add_release(&B->count);
        if (ld_acquire(&B->count) < target) {
            const uint64_t t0 = hprsmall::now_ns();
            unsigned polls = 0;
            while (ld_acquire(&B->count) < target) {
                if ((++polls & 63u) == 0) {
                    if (ld_relaxed(&B->err)) { ok = 0; break; }
                    if (hprsmall::now_ns() - t0 > P.budget_ns) {
                        if (atomicExch(&B->err, 1) == 0) B->where = nb;
                        ok = 0;
                        break;
                    }
                }
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Row sums of M against x over the slices this warp owns: f(row, sum) on the lane that owns
// the row.  The gathered vector may have been written by other CTAs of this launch: it is
// read through L2.  Two FMA chains (even / odd steps), then the fixed xor butterfly of the
// single-CTA path, so a row's sum does not depend on the grid size.
template <class F>
__device__ __forceinline__ void grid_rows(const hprsmall::SmallMat &M, const double *x, int gw, int GW, F f)
{
    const int lane = threadIdx.x & 31;
    for (int s = gw; s < M.nslices; s += GW) {
        const int lg = __ldg(M.slg + s);
        const int r0 = __ldg(M.srow + s), r1 = __ldg(M.srow + s + 1);
        const int p0 = __ldg(M.sptr + s) + lane, steps = (__ldg(M.sptr + s + 1) - __ldg(M.sptr + s)) >> 5;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 < steps; k += 2) {
            const int pa = p0 + (k << 5), pb = pa + 32;
            const double va = __ldg(M.val + pa), vb = __ldg(M.val + pb);
            const int ca = HPR_COL(__ldg(M.col + pa), M.cols), cb = HPR_COL(__ldg(M.col + pb), M.cols);
            a0 = fma(va, __ldcg(x + ca), a0);
            a1 = fma(vb, __ldcg(x + cb), a1);
        }
        if (k < steps) {
            const int pa = p0 + (k << 5);
            a0 = fma(__ldg(M.val + pa), __ldcg(x + HPR_COL(__ldg(M.col + pa), M.cols)), a0);
        }
        double sum = steps > 1 ? a0 + a1 : a0;
        for (int o = 1; o < (1 << lg); o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const int row = r0 + (lane >> lg);
        if ((lane & ((1 << lg) - 1)) == 0 && row < r1) f(row, sum);
    }
}

// Fixed-order CTA sums of NV values per thread (xor butterfly in each warp, then warp 0 over
// the NW warp sums in warp order) published as the partials of CTA `rank` of the launch (or
// cluster); red holds NV * NW doubles.
template <int NV>
__device__ __forceinline__ void cta_publish(double (&v)[NV], double *red, double *partials, int G, int rank)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q * NW + w] = v[q];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = lane < NW ? red[q * NW + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) __stcg(partials + q * G + rank, s);
        }
    }
}

// After a barrier: the grid sums of the NV published quantities, the same in every CTA
// (lanes take the CTA sums in a fixed strided order, then a fixed xor butterfly); warp 0
// of the CTA computes them and hands them to g on thread 0.
template <int NV, class Gf>
__device__ __forceinline__ void grid_sums_then(const double *partials, int G, Gf g)
{
    if ((threadIdx.x >> 5) != 0) return;
    const int lane = threadIdx.x & 31;
    double sum[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = 0.0;
        for (int b = lane; b < G; b += 32) t += __ldcg(partials + q * G + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        sum[q] = t;
    }
    if (lane == 0) g(static_cast<const double *>(sum));
}

// Algorithm 2's outer-loop state: thread 0 of every CTA keeps its own copy, and all copies
// stay equal because every CTA sees bitwise the same check sums
struct OuterState {
    int64_t r = 0, nrec = 0, i1e4 = -1;
    double R0 = 0.0, Rprev = 0.0, t1e4 = -1.0;
    double pobj = 0, dobj = 0, errp = 0, errd = 0, gap = 0, kkt = 0;
    int status = 1;                                    // HPR_MAX_ITER
};

// The decisions at a check from its grid sums (thread 0 of a CTA): the merit R~ of eq.
// (def:M), the termination test of Section 4.1, the restart criteria eq. (restart_1)-
// (restart_3) and Algorithm 3's sigma.  CTA (rank) 0 writes the check record.  Returns in
// *restart / *stop whether the inner loop restarts / the solve ends, and the next sigma.
__device__ __forceinline__ void check_decide(const GridArgs &P, OuterState &D, const double *sums, int rank,
                                             int64_t k, int64_t t_all, bool is_r0, bool is_check, double sigma,
                                             double lambda, double elapsed, int *restart, int *stop,
                                             double *sigma_out)
{
    const double S_DX2 = sums[0], S_XX0 = sums[1], S_CX = sums[2], S_BND = sums[3], S_DY2 = sums[4];
    const double S_YY0 = sums[5], S_BY = sums[6], S_RD = sums[7], S_RP = sums[8], S_CROSS = sums[9];
    // ||w - w_hat||_M = 2 ||w - w_bar||_M, eq. (def:M) with T1 = lambda I - A A^*
    const double qm = sigma * lambda * S_DY2 + 2.0 * S_CROSS + S_DX2 / sigma;
    const double Rt = 2.0 * sqrt(qm > 0.0 ? qm : 0.0);
    const bool rec_ok = rank == 0 && D.nrec < P.rec_cap;
    *restart = 0;
    *stop = 0;
    *sigma_out = sigma;
    if (is_r0 && !is_check) {
        D.R0 = Rt;
        D.Rprev = Rt;
        if (rec_ok) {
            hpr_check_record rec{};
            rec.k = k; rec.r = D.r; rec.t = 0; rec.kind = 2; rec.cause = 0;
            rec.sigma = sigma; rec.Rt = D.R0; rec.R0 = D.R0; rec.sigma_next = sigma;
            rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = sigma;
            P.recs[D.nrec] = rec;
        }
        ++D.nrec;
        return;
    }
    if (is_r0) {
        D.R0 = Rt;
        D.Rprev = Rt;
    }
    // termination test of Section 4.1 in the original space
    const double bb = P.beta_b * P.beta_c;
    D.errp = sqrt(S_RP) / (1.0 + P.norm_b);
    D.errd = sqrt(S_RD) / (1.0 + P.norm_c);
    D.pobj = bb * S_CX;
    D.dobj = bb * (S_BY + S_BND);
    D.gap = fabs(D.dobj - D.pobj) / (1.0 + fabs(D.pobj) + fabs(D.dobj));
    D.kkt = fmax(D.errp, fmax(D.errd, D.gap));
    if (D.t1e4 < 0.0 && D.kkt <= 1e-4) {
        D.t1e4 = elapsed;
        D.i1e4 = k + 1;
    }
    int cause = 0;
    double sigma_next = sigma, Dx = 0.0, Dy = 0.0;
    if (!(D.kkt == D.kkt) || !(Rt == Rt) || isinf(D.kkt) || isinf(Rt)) {
        D.status = -6;                                 // HPR_ERR_NUMERIC
        *stop = 1;
    } else if (D.kkt <= P.tol) {
        D.status = 0;
        cause = -1;
        *stop = 1;
    } else if (k + 1 < P.max_iter && P.restart && !is_r0) {
        // restart criteria eq. (restart_1)-(restart_3)
        if (Rt <= P.alpha1 * D.R0) cause = 1;
        else if (Rt <= P.alpha2 * D.R0 && Rt > D.Rprev) cause = 2;
        else if ((double)(t_all + 1) >= P.alpha3 * (double)(k + 1)) cause = 3;
        D.Rprev = Rt;
        *restart = cause != 0;
    }
    if (*restart) {
        // Algorithm 3 with eq. (sigma_T1!=0)
        Dx = sqrt(S_XX0);
        Dy = sqrt(lambda) * sqrt(S_YY0);
        const double ratio = D.errd / D.errp;
        if (P.sigma_update && Dx > 1e-16 && Dx < 1e12 && Dy > 1e-16 && Dy < 1e12 && D.errp > 0.0 &&
            ratio > 1e-8 && ratio < 1e8)
            sigma_next = Dx / Dy;
        else
            sigma_next = P.sigma_update ? 1.0 : sigma;
    }
    if (rec_ok) {
        hpr_check_record rec{};
        rec.k = k; rec.r = D.r; rec.t = t_all; rec.kind = 1 + (is_r0 ? 2 : 0); rec.cause = cause;
        rec.sigma = sigma; rec.err_p = D.errp; rec.err_d = D.errd; rec.err_gap = D.gap; rec.kkt = D.kkt;
        rec.pobj = D.pobj; rec.dobj = D.dobj; rec.Rt = Rt; rec.R0 = D.R0; rec.sigma_next = sigma_next;
        rec.Dx = Dx; rec.Dy = Dy; rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = sigma_next;
        P.recs[D.nrec] = rec;
    }
    ++D.nrec;
    if (*restart) {
        *sigma_out = sigma_next;
        ++D.r;
    }
}

// the results of a persistent solve (CTA 0, thread 0)
__device__ __forceinline__ void write_out(const GridArgs &P, const OuterState &D, int64_t k, double lambda,
                                          int64_t piters, double sigma, double prel, uint64_t t_start,
                                          uint64_t t_power)
{
    double *o = P.out;
    using namespace hprsmall;
    o[SO_ITERS] = (double)k; o[SO_RESTARTS] = (double)D.r; o[SO_STATUS] = (double)D.status;
    o[SO_LAMBDA] = lambda; o[SO_POWER_ITERS] = (double)piters; o[SO_SIGMA] = sigma;
    o[SO_POBJ] = D.pobj; o[SO_DOBJ] = D.dobj; o[SO_ERRP] = D.errp; o[SO_ERRD] = D.errd; o[SO_GAP] = D.gap;
    o[SO_KKT] = D.kkt; o[SO_T1E4] = D.t1e4; o[SO_I1E4] = (double)D.i1e4; o[SO_NREC] = (double)D.nrec;
    o[SO_POWER_S] = 1e-9 * (double)(t_power - t_start);
    o[SO_TOTAL_S] = 1e-9 * (double)(hprsmall::now_ns() - t_start);
    o[SO_POWER_REL] = prel;
}

__global__ void __launch_bounds__(NT) k_solve_grid(GridArgs P)
{
    using hprsmall::now_ns;
    const int tid = threadIdx.x, G = P.G;
    // CTA-minor warp numbering; A^T's slices start half the grid further on, so that the
    // longest slices of A and of A^T do not land in the same CTA
    const int GW = G * NW;
    const int gwA = (tid >> 5) * G + (int)blockIdx.x, gwT = (tid >> 5) * G + ((int)blockIdx.x + G / 2) % G;
    const hprsmall::SmallMat MA = P.A, MT = P.T;
    const int n = P.n, m = P.m;
    double *x = P.x, *x0 = P.x0, *xh = P.xh, *xb = P.xb, *zb = P.zb, *dx = P.dx;
    double *y = P.y, *y0 = P.y0, *yb = P.yb, *dy = P.dy;
    __shared__ double red[NQG * NW];
    __shared__ int s_ok, s_flag;
    __shared__ double sc[4];                  // power method: 1/||w||, lambda_k
    __shared__ double bc_sigma, bc_ha, bc_hb, bc_ils;
    __shared__ int bc_restart, bc_stop;
    __shared__ double sc_in[2];
    int nb = 0;                               // barriers passed
    const uint64_t t_start = now_ns();

    // ---- lambda of T1 = lambda I - A A^* (power method of Section 4.1, counted in the solve
    // time): u in dy, s = A^T w / ||w|| in dx, w = A s in yb
    double lambda = P.lambda_fixed;
    int64_t piters = 0;
    double prel = 0.0;
    if (!(lambda > 0.0)) {
        double p[1] = {0.0};
        for (int i = blockIdx.x * NT + tid; i < m; i += G * NT) {
            const double v = 2.0 * ((double)(hprdev::splitmix64_at(P.seed, (uint64_t)P.perm_r[i]) >> 11) * 0x1.0p-53) - 1.0;
            __stcg(yb + i, v);
            p[0] = fma(v, v, p[0]);
        }
        cta_publish<1>(p, red, P.partials, G, blockIdx.x);
        if (!grid_sync(P, nb++, &s_ok)) return;
        grid_sums_then<1>(P.partials, G, [&](const double *sum) {
            sc[0] = 1.0 / sqrt(sum[0]);
            sc[1] = 0.0;
            s_flag = 0;
        });
        __syncthreads();
        int64_t k = 0;
        for (;;) {
            const double inv = sc[0];
            double q[2] = {0.0, 0.0};
            grid_rows(MT, yb, gwT, GW, [&](int j, double sj) {
                const double t = sj * inv;
                __stcg(dx + j, t);
                q[0] = fma(t, t, q[0]);
            });
            if (!grid_sync(P, nb++, &s_ok)) return;
            grid_rows(MA, dx, gwA, GW, [&](int i, double wi) {
                __stcg(yb + i, wi);
                q[1] = fma(wi, wi, q[1]);
            });
            ++k;
            cta_publish<2>(q, red, P.partials, G, blockIdx.x);
            if (!grid_sync(P, nb++, &s_ok)) return;
            grid_sums_then<2>(P.partials, G, [&](const double *sum) {
                const double l = sum[0], prev = sc[1];
                sc[1] = l;
                if (k > 1) sc[2] = fabs(l - prev) / l;
                if ((k > 1 && fabs(l - prev) <= P.power_tol * l) || k >= P.power_max_iter || !(sum[1] > 0.0))
                    s_flag = 1;
                else
                    sc[0] = 1.0 / sqrt(sum[1]);
            });
            __syncthreads();
            if (s_flag) break;
        }
        lambda = sc[1];
        piters = k;
        prel = k > 1 ? sc[2] : 0.0;
    }
    const uint64_t t_power = now_ns();

    auto set_weights = [&](int64_t tn_) {
        volatile double *v = sc_in;
        v[0] = (double)tn_ + 2.0;
        const double d0 = v[0];
        bc_ha = P.halpern ? 1.0 / d0 : 0.0;
        bc_hb = P.halpern ? (d0 - 1.0) / d0 : 1.0;
    };
    auto set_sigma = [&](double sg) {
        volatile double *v = sc_in;
        bc_sigma = sg;
        v[1] = lambda * sg;
        bc_ils = 1.0 / v[1];
    };
    if (tid == 0) {
        set_sigma(P.sigma0);
        set_weights(0);
    }
    __syncthreads();

    // Algorithm 2 from the origin (Section 4.1): x = x0 = 0, y = y0 = 0
    for (int j = blockIdx.x * NT + tid; j < n; j += G * NT) {
        __stcg(x + j, 0.0);
        __stcg(x0 + j, 0.0);
    }
    for (int i = blockIdx.x * NT + tid; i < m; i += G * NT) {
        __stcg(y + i, 0.0);
        __stcg(y0 + i, 0.0);
    }
    if (!grid_sync(P, nb++, &s_ok)) return;
    int64_t k = 0;
    OuterState D;
    int64_t t_all = 0;
    int64_t to_check = P.check_every;
    int fresh = 0;                                     // 1: first iteration after a restart
#pragma unroll 1
    for (k = 0; k < P.max_iter; ++k) {
        const double sigma = bc_sigma, ha = bc_ha, hb = bc_hb, inv_ls = bc_ils;
        const bool periodic = (--to_check == 0);
        if (periodic) to_check = P.check_every;
        const bool is_check = periodic || (k + 1 == P.max_iter);
        const bool is_r0 = (t_all == 0);
        const bool store = is_check || is_r0;
        double q[NQG] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        // phase X: eq. (update-x), reflection, Halpern step (after a restart: x = x0 = x_bar,
        // y = y_bar, Algorithm 2's w^{r+1,0} = w_bar^{r,tau_r})
        grid_rows(MT, fresh ? yb : y, gwT, GW, [&](int j, double sj) {
            double xj, x0j;
            if (!fresh) {
                xj = __ldcg(x + j);
                x0j = __ldcg(x0 + j);
            } else {
                xj = x0j = __ldcg(xb + j);
                __stcg(x0 + j, x0j);
            }
            const double cj = __ldg(P.c + j), lj = __ldg(P.l + j), uj = __ldg(P.u + j);
            const double v = fma(sigma, sj - cj, xj);
            const double xbj = hprdev::clamp_lu(v, lj, uj);
            const double xhj = fma(2.0, xbj, -xj);
            __stcg(xh + j, xhj);
            __stcg(x + j, fma(hb, P.reflect ? xhj : xbj, ha * x0j));
            if (store) {
                const double zbj = (xbj - v) / sigma, d = xj - xbj, e = xbj - x0j;
                __stcg(xb + j, xbj);
                __stcg(zb + j, zbj);
                __stcg(dx + j, d);
                q[0] = fma(d, d, q[0]);
                q[1] = fma(e, e, q[1]);
                q[2] = fma(cj, xbj, q[2]);
                if (zbj > 0.0) q[3] = fma(zbj, lj, q[3]);
                else if (zbj < 0.0) q[3] = fma(zbj, uj, q[3]);
            }
        });
        if (!grid_sync(P, nb++, &s_ok)) return;
        // the next iteration's weights, by the last thread while the others update y: every
        // thread read this iteration's values before the barrier above (a check iteration sets
        // them after its decisions instead)
        if (!store && tid == NT - 1) set_weights(t_all + 1);
        // phase Y: eq. (update-y-2), projection on D, reflection, Halpern step
        grid_rows(MA, xh, gwA, GW, [&](int i, double qi) {
            double yi, y0i;
            if (!fresh) {
                yi = __ldcg(y + i);
                y0i = __ldcg(y0 + i);
            } else {
                yi = y0i = __ldcg(yb + i);
                __stcg(y0 + i, y0i);
            }
            const double bi = __ldg(P.b + i);
            double ybi = fma(bi - qi, inv_ls, yi);
            if (P.ineq[i]) ybi = hprdev::pos_part(ybi);
            const double yhi = fma(2.0, ybi, -yi);
            __stcg(y + i, fma(hb, P.reflect ? yhi : ybi, ha * y0i));
            if (store) {
                const double d = yi - ybi, e = ybi - y0i;
                __stcg(yb + i, ybi);
                __stcg(dy + i, d);
                q[4] = fma(d, d, q[4]);
                q[5] = fma(e, e, q[5]);
                q[6] = fma(bi, ybi, q[6]);
            }
        });
        fresh = 0;
        if (!grid_sync(P, nb++, &s_ok)) return;
        if (!store) {
            ++t_all;
            continue;
        }
        // the check quantities: residual passes in the original-space weights, <dy, A dx>
        grid_rows(MT, yb, gwT, GW, [&](int j, double sj) {
            const double rj = __ldg(P.wc + j) * (__ldg(P.c + j) - sj - __ldcg(zb + j));
            q[7] = fma(rj, rj, q[7]);
        });
        grid_rows(MA, xb, gwA, GW, [&](int i, double si) {
            double ri = __ldg(P.b + i) - si;
            if (P.ineq[i]) ri = hprdev::pos_part(ri);
            ri *= __ldg(P.wr + i);
            q[8] = fma(ri, ri, q[8]);
        });
        grid_rows(MA, dx, gwA, GW, [&](int i, double si) { q[9] = fma(__ldcg(dy + i), si, q[9]); });
        cta_publish<NQG>(q, red, P.partials, G, blockIdx.x);
        if (!grid_sync(P, nb++, &s_ok)) return;
        grid_sums_then<NQG>(P.partials, G, [&](const double *sums) {
            int rs, stp;
            double sn;
            check_decide(P, D, sums, blockIdx.x, k, t_all, is_r0, is_check, sigma, lambda,
                         1e-9 * (double)(now_ns() - t_start), &rs, &stp, &sn);
            bc_restart = rs;
            bc_stop = stp;
            if (rs) set_sigma(sn);
            set_weights(rs ? 0 : t_all + 1);
        });
        __syncthreads();
        if (bc_stop) {
            ++k;
            break;
        }
        if (bc_restart) {
            t_all = 0;
            fresh = 1;
        } else {
            ++t_all;
        }
    }
    if (blockIdx.x == 0 && tid == 0) write_out(P, D, k, lambda, piters, bc_sigma, prel, t_start, t_power);
}

}  // namespace hprgrid
