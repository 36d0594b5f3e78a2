// Persistent single-CTA solve for LPs small enough that their iterates fit in shared
// memory (the tiny planted family): one CTA of 1024 threads runs the power method and the
// whole of Algorithm 2 -- iterations, checks every check_every iterations, the restart
// criteria, SigmaUpdate (Algorithm 3) and the termination test -- without returning to the
// host, so an iteration costs two block barriers instead of two kernel launches.
//
// One SM is bound by its FP64 issue: the FP64 pipe takes one warp instruction every ~17
// cycles whatever the number of active lanes.  So the kernel works in the multi-CTA path's
// renumbered order on the same sliced-ELL layouts of A and A^T (rows by decreasing length,
// 32-row slices stored column-major): a warp takes whole slices, the rows of a slice have
// similar lengths, and an FP64 instruction rarely idles lanes.  The lane that owns a row
// finishes the row's update (the epilogue) right after its sum, so a phase needs no barrier
// between the SpMV and the update.  Every reduction has a fixed order; reductions involve
// only the warps that own rows.  The decisions are those of the host loop of the multi-CTA
// path, taken by thread 0 and broadcast through shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hprsmall {

constexpr int NT = 1024;
constexpr int NW = NT / 32;

// a sliced-ELL matrix as the multi-CTA path stores it (slice s: rows srow[s] .. srow[s+1]-1,
// L = 2^slg[s] lanes per row, entries sptr[s] .. sptr[s+1]-1 in steps of 32, column-major)
struct SmallMat {
    int nslices;
    int cols;                                // length of the gathered vectors
    int64_t entries;
    const int *srow, *sptr, *col;
    const unsigned char *slg;
    const double *val;
};

struct SmallArgs {
    int m, n;
    SmallMat A, T;                           // A (m rows) and A^T (n rows), renumbered
    const unsigned char *ineq;               // renumbered row i of A belongs to A2
    const double *b, *c, *l, *u, *wr, *wc;   // scaled data and residual weights, renumbered
    double beta_b, beta_c, norm_b, norm_c;
    // options
    double tol, alpha1, alpha2, alpha3, sigma0, lambda_fixed, power_tol;
    int64_t max_iter, check_every, power_max_iter;
    uint64_t seed;
    int restart, sigma_update, halpern, reflect;
    int mat_smem;                            // 1: copy both layouts into shared memory too
    const int *perm_r;                       // original row of renumbered row i (start vector)
    // outputs: the last w_bar, renumbered (the multi-CTA path's back-map reads them)
    double *xbar_out, *ybar_out, *zbar_out;
    hpr_check_record *recs;
    int rec_cap;
    double *out;                             // SMALL_OUT values, below
};

enum {
    SO_ITERS, SO_RESTARTS, SO_STATUS, SO_LAMBDA, SO_POWER_ITERS, SO_SIGMA, SO_POBJ, SO_DOBJ, SO_ERRP,
    SO_ERRD, SO_GAP, SO_KKT, SO_T1E4, SO_I1E4, SO_NREC, SO_POWER_S, SO_TOTAL_S, SO_POWER_REL, SO_LEN
};

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// warps that own rows of a matrix with `nslices` slices (warp w takes slices w, w + NW, ...)
__host__ __device__ __forceinline__ int owner_warps(int nslices)
{
    return nslices < NW ? nslices : NW;
}

// Row sums of M against x: for every row, f(row, sum) on the lane that owns the row.
// A lane accumulates the even and the odd steps of its slice in two FMA chains (in step
// order) and adds them; the L lanes of a row are then added by a fixed xor butterfly.
template <class F>
__device__ __forceinline__ void sell_rows(const SmallMat &M, const double *x, F f)
{
    const int lane = threadIdx.x & 31;
    for (int s = threadIdx.x >> 5; s < M.nslices; s += NW) {
        const int lg = M.slg[s];
        const int r0 = M.srow[s], r1 = M.srow[s + 1];
        const int p0 = M.sptr[s] + lane, steps = (M.sptr[s + 1] - M.sptr[s]) >> 5;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 < steps; k += 2) {
            const int pa = p0 + (k << 5), pb = pa + 32;
            a0 = fma(M.val[pa], x[HPR_COL(M.col[pa], M.cols)], a0);
            a1 = fma(M.val[pb], x[HPR_COL(M.col[pb], M.cols)], a1);
        }
        if (k < steps) {
            const int pa = p0 + (k << 5);
            a0 = fma(M.val[pa], x[HPR_COL(M.col[pa], M.cols)], a0);
        }
        double sum = steps > 1 ? a0 + a1 : a0;
        for (int o = 1; o < (1 << lg); o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const int row = r0 + (lane >> lg);
        if ((lane & ((1 << lg) - 1)) == 0 && row < r1) f(row, sum);
    }
}

// Fixed-order sums over the CTA of NV values per thread when only warps < nact hold nonzero
// values: an xor butterfly inside each of those warps, then warp 0 over their sums in warp
// order.  red holds NV * 32 doubles; the sums land in outv[0 .. NV-1] (shared memory),
// valid for every thread on return.
template <int NV>
__device__ __forceinline__ void cta_sums(double (&v)[NV], int nact, double *red, double *outv)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < nact) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NV; ++q) red[q * 32 + w] = v[q];
        }
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = lane < nact ? red[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) outv[q] = s;
        }
    }
    __syncthreads();
}

// The same fixed-order sums, handed to g(sums) on thread 0 before the closing barrier: g
// takes a decision and publishes it through shared memory, so that no other warp spends
// FP64 issue slots on it.
template <int NV, class G>
__device__ __forceinline__ void cta_sums_then(double (&v)[NV], int nact, double *red, G g)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < nact) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NV; ++q) red[q * 32 + w] = v[q];
        }
    }
    __syncthreads();
    if (w == 0) {
        double sum[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = lane < nact ? red[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            sum[q] = t;
        }
        if (lane == 0) g(static_cast<const double *>(sum));
    }
    __syncthreads();
}

// power method on A A^* (Section 4.1): u0 from SplitMix64(seed) at each row's original
// index, normalised; s = A^T u, lambda = ||s||^2, stop when |lambda_k - lambda_{k-1}| <=
// tol lambda_k or after power_max_iter steps; u = A s / ||A s||.  w (m, u unnormalised) and
// s (n) are shared-memory scratch; sc holds the broadcast scalars.  A step computes
// s = (A^T w) / ||w|| (the normalisation applied in the row sums) and w' = A s, then sums
// ||s||^2 and ||w'||^2 in one reduction whose thread 0 takes the decisions: three barriers
// a step and no FP64 work outside the warps that own rows.  (The last step's A s is not
// needed; it keeps the step uniform.)
__device__ double power_small(const SmallArgs &P, double *w, double *s, double *red, double *sc, int *flag,
                              int64_t *iters, double *rel_change)
{
    const int tid = threadIdx.x;
    const int act_m = owner_warps((P.m + 31) / 32), actA = owner_warps(P.A.nslices),
              actT = owner_warps(P.T.nslices);
    double p[2] = {0.0, 0.0};
    for (int i = tid; i < P.m; i += NT) {
        const uint64_t o = (uint64_t)P.perm_r[i];
        const double v = 2.0 * ((double)(hprdev::splitmix64_at(P.seed, o) >> 11) * 0x1.0p-53) - 1.0;
        w[i] = v;
        p[0] = fma(v, v, p[0]);
    }
    // sc[0]: 1 / ||w||, sc[1]: lambda_k; flag: stop
    cta_sums<2>(p, act_m, red, sc);
    if (tid == 0) {
        sc[0] = 1.0 / sqrt(((volatile double *)sc)[0]);
        *flag = 0;
    }
    __syncthreads();
    const int act = actA > actT ? actA : actT;
    double lam = 0.0;
    int64_t k = 0;
    for (;;) {
        const double inv = sc[0];
        double q[2] = {0.0, 0.0};
        sell_rows(P.T, w, [&](int j, double sj) {
            const double t = sj * inv;
            s[j] = t;
            q[0] = fma(t, t, q[0]);
        });
        __syncthreads();
        sell_rows(P.A, s, [&](int i, double wi) {
            w[i] = wi;
            q[1] = fma(wi, wi, q[1]);
        });
        ++k;
        cta_sums_then<2>(q, act, red, [&](const double *sum) {
            const double l = sum[0], prev = sc[1];
            sc[1] = l;
            if (k > 1) sc[2] = fabs(l - prev) / l;
            if ((k > 1 && fabs(l - prev) <= P.power_tol * l) || k >= P.power_max_iter || !(sum[1] > 0.0))
                *flag = 1;
            else
                sc[0] = 1.0 / sqrt(sum[1]);
        });
        if (*flag) break;
    }
    lam = sc[1];
    *iters = k;
    *rel_change = k > 1 ? sc[2] : 0.0;
    return lam;
}

// The power method alone in one CTA, for LPs that fit one SM but whose iterations run on
// the multi-CTA path (the FP32 form, tracing, a time limit, ...): w (m) and s (n) in
// shared memory; out = {lambda, steps, last relative change of lambda}.
__global__ void __launch_bounds__(NT) k_power_small(const SmallArgs *__restrict__ args, double *out)
{
    extern __shared__ double sh[];
    const SmallArgs P = *args;
    __shared__ double red[2 * 32];
    __shared__ double sc[3];
    __shared__ int flag;
    int64_t iters = 0;
    double rel = 0.0;
    const double lam = power_small(P, sh, sh + P.m, red, sc, &flag, &iters, &rel);
    if (threadIdx.x == 0) {
        out[0] = lam;
        out[1] = (double)iters;
        out[2] = rel;
    }
}

// Shared memory: n-vectors x, x0, xhat, xbar, zbar, dx; m-vectors y, y0, ybar, dy; with the
// matrices: the values of A's and A^T's layouts, then their column indices and slice
// tables, then their lane counts.
inline size_t small_vec_bytes(int m, int n)
{
    return sizeof(double) * (6 * (size_t)n + 4 * (size_t)m);
}

inline size_t small_smem_bytes(int m, int n, const SmallMat &A, const SmallMat &T, bool mat)
{
    size_t b = small_vec_bytes(m, n);
    if (mat) {
        b += sizeof(double) * (size_t)(A.entries + T.entries);
        b += sizeof(int) * ((size_t)(A.entries + T.entries) + 2 * (size_t)(A.nslices + 1) + 2 * (size_t)(T.nslices + 1));
        b += (size_t)(A.nslices + T.nslices);
        b = (b + 15) & ~(size_t)15;
    }
    return b;
}

// copy a layout into shared memory at (dv, di, db); returns the shared copy
__device__ SmallMat stage_mat(const SmallMat &M, double *&dv, int *&di, unsigned char *&db)
{
    SmallMat S = M;
    const int tid = threadIdx.x;
    for (int64_t p = tid; p < M.entries; p += NT) dv[p] = M.val[p];
    S.val = dv;
    dv += M.entries;
    for (int64_t p = tid; p < M.entries; p += NT) di[p] = M.col[p];
    S.col = di;
    di += M.entries;
    for (int s = tid; s <= M.nslices; s += NT) {
        di[s] = M.srow[s];
        di[M.nslices + 1 + s] = M.sptr[s];
    }
    S.srow = di;
    S.sptr = di + M.nslices + 1;
    di += 2 * (M.nslices + 1);
    for (int s = tid; s < M.nslices; s += NT) db[s] = M.slg[s];
    S.slg = db;
    db += M.nslices;
    return S;
}

// one LP per CTA: block b solves the LP of args[b] (a solo solve launches one block; a batch
// of LPs that all fit launches one block per LP; 1024 threads a block, so at most two
// share an SM)
__global__ void __launch_bounds__(NT) k_solve_small(const SmallArgs *__restrict__ args)
{
    SmallArgs P = args[blockIdx.x];
    extern __shared__ double sh[];
    const int n = P.n, m = P.m, tid = threadIdx.x;
    double *x = sh, *x0 = x + n, *xh = x0 + n, *xb = xh + n, *zb = xb + n, *dx = zb + n;
    double *y = dx + n, *y0 = y + m, *yb = y0 + m, *dy = yb + m;
    if (P.mat_smem) {                    // both layouts into shared memory as well
        double *dv = dy + m;
        int *di = reinterpret_cast<int *>(dv + P.A.entries + P.T.entries);
        unsigned char *db = reinterpret_cast<unsigned char *>(
            di + P.A.entries + P.T.entries + 2 * (P.A.nslices + 1) + 2 * (P.T.nslices + 1));
        P.A = stage_mat(P.A, dv, di, db);
        P.T = stage_mat(P.T, dv, di, db);
        __syncthreads();
    }
    const SmallMat MA = P.A, MT = P.T;
    const int actA = owner_warps(MA.nslices), actT = owner_warps(MT.nslices);
    const int act = actA > actT ? actA : actT;
    __shared__ double red[10 * 32];
    __shared__ double sums[10];
    __shared__ double sc[3];
    __shared__ int pflag;
    __shared__ double sc_in[2];
    __shared__ double bc_sigma, bc_ha, bc_hb, bc_ils;    // this iteration's scalars (thread 0 sets them)
    __shared__ int bc_restart, bc_stop;
    const uint64_t t_start = now_ns();

    // ---- lambda of T1 = lambda I - A A^* (power method, counted in the solve time)
    double lambda = P.lambda_fixed;
    int64_t piters = 0;
    double prel = 0.0;
    if (!(lambda > 0.0)) lambda = power_small(P, yb, x, red, sc, &pflag, &piters, &prel);
    const uint64_t t_power = now_ns();

    // ---- origin start, sigma_0 (Section 4.1)
    for (int j = tid; j < n; j += NT) x[j] = x0[j] = 0.0;
    for (int i = tid; i < m; i += NT) y[i] = y0[i] = 0.0;
    // The Halpern weights of the coming iteration and, after a change of sigma, 1/(lambda
    // sigma) are computed by one thread (FP64 division is costly on this part; its inputs pass
    // through volatile shared memory so that the divisions cannot be hoisted into every thread).
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

    // the host loop's state, kept by thread 0 (decisions broadcast through shared memory)
    int64_t k = 0, r = 0, nrec = 0, i1e4 = -1;
    double R0 = 0.0, Rprev = 0.0, t1e4 = -1.0;
    double pobj = 0, dobj = 0, errp = 0, errd = 0, gap = 0, kkt = 0;
    int status = 1;                                    // HPR_MAX_ITER
    int64_t t_all = 0;                                 // every thread's copy of t
    int64_t to_check = P.check_every;                  // countdown to the next periodic check
#pragma unroll 1
    for (k = 0; k < P.max_iter; ++k) {
        const double sigma = bc_sigma, ha = bc_ha, hb = bc_hb, inv_ls = bc_ils;
        const bool periodic = (--to_check == 0);
        if (periodic) to_check = P.check_every;
        const bool is_check = periodic || (k + 1 == P.max_iter);
        const bool is_r0 = (t_all == 0);
        const bool store = is_check || is_r0;
        // partial sums of the check quantities (indices as in the reduction below)
        double q[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        // Compiler memory barriers keep each phase's loads and stores in place: without them
        // the compiler's reordering across the phases doubled the time of an iteration.
        asm volatile("" ::: "memory");
        // phase X: eq. (update-x), reflection, Halpern step, on the lane that owns column j
        sell_rows(MT, y, [&](int j, double sj) {
            const double xj = x[j], cj = __ldg(P.c + j), lj = __ldg(P.l + j), uj = __ldg(P.u + j);
            const double v = fma(sigma, sj - cj, xj);
            const double xbj = hprdev::clamp_lu(v, lj, uj);
            const double xhj = fma(2.0, xbj, -xj);
            xh[j] = xhj;
            x[j] = fma(hb, P.reflect ? xhj : xbj, ha * x0[j]);
            if (store) {
                const double zbj = (xbj - v) / sigma, d = xj - xbj, e = xbj - x0[j];
                xb[j] = xbj;
                zb[j] = zbj;
                dx[j] = d;
                q[0] = fma(d, d, q[0]);
                q[1] = fma(e, e, q[1]);
                q[2] = fma(cj, xbj, q[2]);
                if (zbj > 0.0) q[3] = fma(zbj, lj, q[3]);
                else if (zbj < 0.0) q[3] = fma(zbj, uj, q[3]);
            }
        });
        __syncthreads();
        asm volatile("" ::: "memory");
        // the next iteration's weights, by the last thread while the others update y (every
        // thread read this iteration's values before the barrier above); a check iteration
        // sets them after its decisions instead
        if (!store && tid == NT - 1) set_weights(t_all + 1);
        // phase Y: eq. (update-y-2), projection on D, reflection, Halpern step
        sell_rows(MA, xh, [&](int i, double qi) {
            const double yi = y[i], bi = __ldg(P.b + i);
            double ybi = fma(bi - qi, inv_ls, yi);
            if (P.ineq[i]) ybi = hprdev::pos_part(ybi);
            const double yhi = fma(2.0, ybi, -yi);
            y[i] = fma(hb, P.reflect ? yhi : ybi, ha * y0[i]);
            if (store) {
                const double d = yi - ybi, e = ybi - y0[i];
                yb[i] = ybi;
                dy[i] = d;
                q[4] = fma(d, d, q[4]);
                q[5] = fma(e, e, q[5]);
                q[6] = fma(bi, ybi, q[6]);
            }
        });
        __syncthreads();
        asm volatile("" ::: "memory");
        if (!store) {
            ++t_all;
            continue;
        }
        // the check quantities: residual passes and fixed-order sums
        sell_rows(MT, yb, [&](int j, double sj) {           // dual residual, original space
            const double rj = __ldg(P.wc + j) * (__ldg(P.c + j) - sj - zb[j]);
            q[7] = fma(rj, rj, q[7]);
        });
        sell_rows(MA, xb, [&](int i, double si) {           // primal residual, original space
            double ri = __ldg(P.b + i) - si;
            if (P.ineq[i]) ri = hprdev::pos_part(ri);
            ri *= __ldg(P.wr + i);
            q[8] = fma(ri, ri, q[8]);
        });
        sell_rows(MA, dx, [&](int i, double si) { q[9] = fma(dy[i], si, q[9]); });   // <dy, A dx>
        cta_sums<10>(q, act, red, sums);
        if (tid == 0) {
            const double S_DX2 = sums[0], S_XX0 = sums[1], S_CX = sums[2], S_BND = sums[3], S_DY2 = sums[4];
            const double S_YY0 = sums[5], S_BY = sums[6], S_RD = sums[7], S_RP = sums[8], S_CROSS = sums[9];
            // ||w - w_hat||_M = 2 ||w - w_bar||_M, eq. (def:M) with T1 = lambda I - A A^*
            const double qm = sigma * lambda * S_DY2 + 2.0 * S_CROSS + S_DX2 / sigma;
            const double Rt = 2.0 * sqrt(qm > 0.0 ? qm : 0.0);
            const double elapsed = 1e-9 * (double)(now_ns() - t_start);
            bc_restart = 0;
            bc_stop = 0;
            if (is_r0 && !is_check) {
                R0 = Rt;
                Rprev = Rt;
                if (nrec < P.rec_cap) {
                    hpr_check_record rec{};
                    rec.k = k; rec.r = r; rec.t = 0; rec.kind = 2; rec.cause = 0;
                    rec.sigma = sigma; rec.Rt = R0; rec.R0 = R0; rec.sigma_next = sigma;
                    rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = sigma;
                    P.recs[nrec] = rec;
                }
                ++nrec;
            } else {
                if (is_r0) {
                    R0 = Rt;
                    Rprev = Rt;
                }
                // termination test of Section 4.1 in the original space
                const double bb = P.beta_b * P.beta_c;
                errp = sqrt(S_RP) / (1.0 + P.norm_b);
                errd = sqrt(S_RD) / (1.0 + P.norm_c);
                pobj = bb * S_CX;
                dobj = bb * (S_BY + S_BND);
                gap = fabs(dobj - pobj) / (1.0 + fabs(pobj) + fabs(dobj));
                kkt = fmax(errp, fmax(errd, gap));
                if (t1e4 < 0.0 && kkt <= 1e-4) {
                    t1e4 = elapsed;
                    i1e4 = k + 1;
                }
                int cause = 0;
                double sigma_next = sigma, Dx = 0.0, Dy = 0.0;
                if (!(kkt == kkt) || !(Rt == Rt) || isinf(kkt) || isinf(Rt)) {
                    status = -6;                       // HPR_ERR_NUMERIC
                    bc_stop = 1;
                } else if (kkt <= P.tol) {
                    status = 0;
                    cause = -1;
                    bc_stop = 1;
                } else if (k + 1 < P.max_iter && P.restart && !is_r0) {
                    // restart criteria eq. (restart_1)-(restart_3)
                    if (Rt <= P.alpha1 * R0) cause = 1;
                    else if (Rt <= P.alpha2 * R0 && Rt > Rprev) cause = 2;
                    else if ((double)(t_all + 1) >= P.alpha3 * (double)(k + 1)) cause = 3;
                    Rprev = Rt;
                    bc_restart = cause != 0;
                }
                if (bc_restart) {
                    // Algorithm 3 with eq. (sigma_T1!=0)
                    Dx = sqrt(S_XX0);
                    Dy = sqrt(lambda) * sqrt(S_YY0);
                    const double ratio = errd / errp;
                    if (P.sigma_update && Dx > 1e-16 && Dx < 1e12 && Dy > 1e-16 && Dy < 1e12 && errp > 0.0 &&
                        ratio > 1e-8 && ratio < 1e8)
                        sigma_next = Dx / Dy;
                    else
                        sigma_next = P.sigma_update ? 1.0 : sigma;
                }
                if (nrec < P.rec_cap) {
                    hpr_check_record rec{};
                    rec.k = k; rec.r = r; rec.t = t_all; rec.kind = 1 + (is_r0 ? 2 : 0); rec.cause = cause;
                    rec.sigma = sigma; rec.err_p = errp; rec.err_d = errd; rec.err_gap = gap; rec.kkt = kkt;
                    rec.pobj = pobj; rec.dobj = dobj; rec.Rt = Rt; rec.R0 = R0; rec.sigma_next = sigma_next;
                    rec.Dx = Dx; rec.Dy = Dy; rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = sigma_next;
                    P.recs[nrec] = rec;
                }
                ++nrec;
                if (bc_restart) {
                    set_sigma(sigma_next);
                    ++r;
                }
            }
            set_weights(bc_restart ? 0 : t_all + 1);
        }
        __syncthreads();
        if (bc_stop) {
            ++k;
            break;
        }
        if (bc_restart) {
            // w^{r+1,0} = w_bar: new anchor
            for (int j = tid; j < n; j += NT) x[j] = x0[j] = xb[j];
            for (int i = tid; i < m; i += NT) y[i] = y0[i] = yb[i];
            t_all = 0;
        } else {
            ++t_all;
        }
        __syncthreads();
    }
    // the last w_bar (renumbered, for the multi-CTA path's back-map)
    for (int j = tid; j < n; j += NT) {
        P.xbar_out[j] = xb[j];
        P.zbar_out[j] = zb[j];
    }
    for (int i = tid; i < m; i += NT) P.ybar_out[i] = yb[i];
    if (tid == 0) {
        double *o = P.out;
        o[SO_ITERS] = (double)k; o[SO_RESTARTS] = (double)r; o[SO_STATUS] = (double)status;
        o[SO_LAMBDA] = lambda; o[SO_POWER_ITERS] = (double)piters; o[SO_SIGMA] = bc_sigma;
        o[SO_POBJ] = pobj; o[SO_DOBJ] = dobj; o[SO_ERRP] = errp; o[SO_ERRD] = errd; o[SO_GAP] = gap;
        o[SO_KKT] = kkt; o[SO_T1E4] = t1e4; o[SO_I1E4] = (double)i1e4; o[SO_NREC] = (double)nrec;
        o[SO_POWER_S] = 1e-9 * (double)(t_power - t_start);
        o[SO_TOTAL_S] = 1e-9 * (double)(now_ns() - t_start);
        o[SO_POWER_REL] = prel;
    }
}

}  // namespace hprsmall
