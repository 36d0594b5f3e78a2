// Persistent single-CTA solve for LPs small enough that their iterates fit in shared
// memory (the tiny planted family): one CTA of 1024 threads runs the power method and the
// whole of Algorithm 2 -- iterations, checks every check_every iterations, the restart
// criteria, SigmaUpdate (Algorithm 3) and the termination test -- without returning to the
// host, so an iteration costs a few block barriers instead of two kernel launches.
// The scaled CSR of A and A^T are read from global memory (they stay in L1); the iterates
// live in shared memory.  Rows are summed in CSR order by one thread each; every reduction
// is a fixed-order block sum.  The decisions are those of the host loop of the multi-CTA
// path, taken by thread 0 and broadcast through shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hprsmall {

constexpr int NT = 1024;

struct SmallArgs {
    int m, m1, n;
    const int *rp, *ci, *trp, *tci;          // scaled A and A^T (original order)
    const double *val, *tval;
    const double *b, *c, *l, *u, *wr, *wc;   // scaled data and residual weights
    double beta_b, beta_c, norm_b, norm_c;
    // options
    double tol, alpha1, alpha2, alpha3, sigma0, lambda_fixed, power_tol;
    int64_t max_iter, check_every, power_max_iter;
    uint64_t seed;
    int restart, sigma_update, halpern, reflect;
    int LA, LT;                              // lanes per row of A's and A^T's row sums
    int nnz, mat_smem;                       // 1: copy A and A^T into shared memory too
    // outputs: final iterates scattered into the renumbered order of the multi-CTA path
    const int *perm_r, *perm_c;
    double *xbar_out, *ybar_out, *zbar_out;
    hpr_check_record *recs;
    int rec_cap;
    double *out;                             // SMALL_OUT values, below
};

enum {
    SO_ITERS, SO_RESTARTS, SO_STATUS, SO_LAMBDA, SO_POWER_ITERS, SO_SIGMA, SO_POBJ, SO_DOBJ, SO_ERRP,
    SO_ERRD, SO_GAP, SO_KKT, SO_T1E4, SO_I1E4, SO_NREC, SO_POWER_S, SO_TOTAL_S, SO_LEN
};

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// fixed-order sum over the CTA: warp trees, then warp 0 over the 32 warp sums
__device__ __forceinline__ double cta_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = red[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// out[r] = sum over row r of val * x, for all rows: L lanes per row (a power of two <= 32),
// lane q taking entries q, q + L, ... of the row in order, then a fixed xor-tree over the
// L lanes; every thread takes part (the loop count is the same for all), then a barrier.
__device__ __forceinline__ void row_sums(const int *rp, const int *ci, const double *val, int rows, int L,
                                         const double *x, double *out)
{
    const int per = NT / L, q = threadIdx.x & (L - 1);
    for (int base = 0; base < rows; base += per) {
        const int r = base + threadIdx.x / L;
        double s = 0.0;
        if (r < rows)
            for (int p = rp[r] + q, pe = rp[r + 1]; p < pe; p += L) s = fma(val[p], x[ci[p]], s);
        for (int o = 1; o < L; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (q == 0 && r < rows) out[r] = s;
    }
    __syncthreads();
}

// power method on A A^* (Section 4.1): u0 from SplitMix64(seed), normalised; s = A^T u,
// lambda = ||s||^2, stop when |lambda_k - lambda_{k-1}| <= tol lambda_k or after
// power_max_iter steps; u = A s / ||A s||.  u, w (m) and s (n) are shared-memory scratch.
__device__ double power_small(const SmallArgs &A, double *u, double *w, double *s, double *red,
                              int64_t *iters)
{
    const int tid = threadIdx.x;
    double p = 0.0;
    for (int i = tid; i < A.m; i += NT) {
        const double v = 2.0 * ((double)(hprdev::splitmix64_at(A.seed, (uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
        u[i] = v;
        p += v * v;
    }
    cta_sum(p, red);
    if (tid == 0) {                      // one thread (inputs reloaded through volatile shared memory so
        const double v = ((volatile double *)red)[32];   // that the costly FP64 divide and root are
        red[33] = 1.0 / sqrt(v);                         // not replicated into every thread)
    }
    __syncthreads();
    const double inv0 = red[33];
    for (int i = tid; i < A.m; i += NT) u[i] *= inv0;
    __syncthreads();
    double lam = 0.0, lam_prev = 0.0;
    int64_t k = 0;
    for (;;) {
        row_sums(A.trp, A.tci, A.tval, A.n, A.LT, u, s);
        double q = 0.0;
        for (int j = tid; j < A.n; j += NT) q += s[j] * s[j];
        lam = cta_sum(q, red);
        ++k;
        if (k > 1 && fabs(lam - lam_prev) <= A.power_tol * lam) break;
        lam_prev = lam;
        row_sums(A.rp, A.ci, A.val, A.m, A.LA, s, w);
        double q2 = 0.0;
        for (int i = tid; i < A.m; i += NT) q2 += w[i] * w[i];
        const double w2 = cta_sum(q2, red);
        if (!(w2 > 0.0) || k >= A.power_max_iter) break;
        if (tid == 0) red[33] = 1.0 / sqrt(((volatile double *)red)[32]);
        __syncthreads();
        const double inv = red[33];
        for (int i = tid; i < A.m; i += NT) u[i] = w[i] * inv;
        __syncthreads();
    }
    *iters = k;
    return lam;
}

// Shared memory: n-vectors x, x0, xhat, xbar, zbar, dx, t_n; m-vectors y, y0, ybar, dy, t_m, t_m2;
// with the matrices: the values of A and A^T, then their row pointers and column indices.
inline size_t small_smem_bytes(int m, int n, int64_t nnz, bool mat)
{
    size_t b = sizeof(double) * (7 * (size_t)n + 6 * (size_t)m);
    if (mat) b += sizeof(double) * 2 * (size_t)nnz + sizeof(int) * ((size_t)m + (size_t)n + 2 + 2 * (size_t)nnz);
    return b;
}

__global__ void __launch_bounds__(NT) k_solve_small(SmallArgs Ain)
{
    SmallArgs A = Ain;
    extern __shared__ double sh[];
    const int n = A.n, m = A.m, tid = threadIdx.x;
    double *x = sh, *x0 = x + n, *xh = x0 + n, *xb = xh + n, *zb = xb + n, *dx = zb + n, *tn = dx + n;
    double *y = tn + n, *y0 = y + m, *yb = y0 + m, *dy = yb + m, *tm = dy + m, *tm2 = tm + m;
    if (A.mat_smem) {                    // A and A^T into shared memory as well
        double *sv = tm2 + m, *stv = sv + A.nnz;
        int *srp = reinterpret_cast<int *>(stv + A.nnz), *strp = srp + m + 1, *sci = strp + n + 1,
            *stci = sci + A.nnz;
        for (int p = tid; p < A.nnz; p += NT) {
            sv[p] = A.val[p];
            stv[p] = A.tval[p];
            sci[p] = A.ci[p];
            stci[p] = A.tci[p];
        }
        for (int i = tid; i <= m; i += NT) srp[i] = A.rp[i];
        for (int j = tid; j <= n; j += NT) strp[j] = A.trp[j];
        A.val = sv; A.tval = stv; A.rp = srp; A.trp = strp; A.ci = sci; A.tci = stci;
        __syncthreads();
    }
    __shared__ double red[34];
    __shared__ double sc_in[2];
    __shared__ double bc_sigma, bc_ha, bc_hb, bc_ils;    // this iteration's scalars (thread 0 sets them)
    __shared__ int bc_restart, bc_stop;
    const uint64_t t_start = now_ns();

    // ---- lambda of T1 = lambda I - A A^* (power method, counted in the solve time)
    double lambda = A.lambda_fixed;
    int64_t piters = 0;
    if (!(lambda > 0.0)) lambda = power_small(A, y, yb, x, red, &piters);
    const uint64_t t_power = now_ns();

    // ---- origin start, sigma_0 (Section 4.1)
    for (int j = tid; j < n; j += NT) x[j] = x0[j] = 0.0;
    for (int i = tid; i < m; i += NT) y[i] = y0[i] = 0.0;
    // sigma, 1/(lambda sigma) and the Halpern weights of the coming iteration, computed by
    // thread 0 only (FP64 division is costly on this part)
    // (thread 0 only: its inputs pass through volatile shared memory so that the divisions
    // cannot be hoisted into every thread)
    auto next_scalars = [&](int64_t tn_) {
        volatile double *v = sc_in;
        v[0] = (double)tn_ + 2.0;
        v[1] = lambda * bc_sigma;
        const double d0 = v[0], d1 = v[1];
        bc_ils = 1.0 / d1;
        bc_ha = A.halpern ? 1.0 / d0 : 0.0;
        bc_hb = A.halpern ? (d0 - 1.0) / d0 : 1.0;
    };
    if (tid == 0) {
        bc_sigma = A.sigma0;
        next_scalars(0);
    }
    __syncthreads();

    // the host loop's state, kept by thread 0 (decisions broadcast through shared memory)
    int64_t k = 0, r = 0, nrec = 0, i1e4 = -1;
    double R0 = 0.0, Rprev = 0.0, t1e4 = -1.0;
    double pobj = 0, dobj = 0, errp = 0, errd = 0, gap = 0, kkt = 0;
    int status = 1;                                    // HPR_MAX_ITER
    int64_t t_all = 0;                                 // every thread's copy of t
    int64_t to_check = A.check_every;                  // countdown to the next periodic check
#pragma unroll 1
    for (k = 0; k < A.max_iter; ++k) {
        const double sigma = bc_sigma, ha = bc_ha, hb = bc_hb, inv_ls = bc_ils;
        const bool periodic = (--to_check == 0);
        if (periodic) to_check = A.check_every;
        const bool is_check = periodic || (k + 1 == A.max_iter);
        const bool is_r0 = (t_all == 0);
        const bool store = is_check || is_r0;
        double p_dx2 = 0, p_xx0 = 0, p_cx = 0, p_bnd = 0, p_dy2 = 0, p_yy0 = 0, p_by = 0;
        // Compiler memory barriers keep each phase's loads and stores in place: without them
        // the compiler's reordering across the phases doubled the time of an iteration
        // (measured: 11.4 against 5.7 microseconds on the tiny planted LP).
        asm volatile("" ::: "memory");
        // phase X: eq. (update-x), reflection, Halpern step
        row_sums(A.trp, A.tci, A.tval, n, A.LT, y, tn);
        asm volatile("" ::: "memory");
        // the next iteration's scalars, by the last thread while the others update x (every
        // thread read this iteration's values before the barrier above); a check iteration
        // sets them after its decisions instead
        if (!store && tid == NT - 1) next_scalars(t_all + 1);
        for (int j = tid; j < n; j += NT) {
            const double sj = tn[j];
            const double xj = x[j], cj = __ldg(A.c + j);
            const double v = fma(sigma, sj - cj, xj);
            const double xbj = fmin(fmax(v, __ldg(A.l + j)), __ldg(A.u + j));
            const double xhj = fma(2.0, xbj, -xj);
            xh[j] = xhj;
            x[j] = fma(hb, A.reflect ? xhj : xbj, ha * x0[j]);
            if (store) {
                const double zbj = (xbj - v) / sigma, d = xj - xbj;
                xb[j] = xbj;
                zb[j] = zbj;
                dx[j] = d;
                p_dx2 = fma(d, d, p_dx2);
                p_xx0 = fma(xbj - x0[j], xbj - x0[j], p_xx0);
                p_cx = fma(cj, xbj, p_cx);
                if (zbj > 0.0) p_bnd = fma(zbj, __ldg(A.l + j), p_bnd);
                else if (zbj < 0.0) p_bnd = fma(zbj, __ldg(A.u + j), p_bnd);
            }
        }
        __syncthreads();
        asm volatile("" ::: "memory");
        // phase Y: eq. (update-y-2), projection on D, reflection, Halpern step
        row_sums(A.rp, A.ci, A.val, m, A.LA, xh, tm);
        asm volatile("" ::: "memory");
        for (int i = tid; i < m; i += NT) {
            const double qi = tm[i];
            const double yi = y[i], bi = __ldg(A.b + i);
            double ybi = fma(bi - qi, inv_ls, yi);
            if (i >= A.m1) ybi = fmax(ybi, 0.0);
            const double yhi = fma(2.0, ybi, -yi);
            y[i] = fma(hb, A.reflect ? yhi : ybi, ha * y0[i]);
            if (store) {
                const double d = yi - ybi;
                yb[i] = ybi;
                dy[i] = d;
                p_dy2 = fma(d, d, p_dy2);
                p_yy0 = fma(ybi - y0[i], ybi - y0[i], p_yy0);
                p_by = fma(bi, ybi, p_by);
            }
        }
        __syncthreads();
        if (!store) {
            ++t_all;
            continue;
        }
        // the check quantities: residual passes and fixed-order sums
        double p_rd = 0, p_rp = 0, p_cross = 0;
        row_sums(A.trp, A.tci, A.tval, n, A.LT, yb, tn);
        row_sums(A.rp, A.ci, A.val, m, A.LA, xb, tm);
        row_sums(A.rp, A.ci, A.val, m, A.LA, dx, tm2);
        for (int j = tid; j < n; j += NT) {
            const double rj = __ldg(A.wc + j) * (__ldg(A.c + j) - tn[j] - zb[j]);
            p_rd = fma(rj, rj, p_rd);
        }
        for (int i = tid; i < m; i += NT) {
            double ri = __ldg(A.b + i) - tm[i];
            if (i >= A.m1) ri = fmax(ri, 0.0);
            ri *= __ldg(A.wr + i);
            p_rp = fma(ri, ri, p_rp);
            p_cross = fma(dy[i], tm2[i], p_cross);
        }
        const double S_DX2 = cta_sum(p_dx2, red), S_XX0 = cta_sum(p_xx0, red), S_CX = cta_sum(p_cx, red);
        const double S_BND = cta_sum(p_bnd, red), S_DY2 = cta_sum(p_dy2, red), S_YY0 = cta_sum(p_yy0, red);
        const double S_BY = cta_sum(p_by, red), S_RD = cta_sum(p_rd, red), S_RP = cta_sum(p_rp, red);
        const double S_CROSS = cta_sum(p_cross, red);
        // ||w - w_hat||_M = 2 ||w - w_bar||_M, eq. (def:M) with T1 = lambda I - A A^*
        const double qm = sigma * lambda * S_DY2 + 2.0 * S_CROSS + S_DX2 / sigma;
        const double Rt = 2.0 * sqrt(qm > 0.0 ? qm : 0.0);
        if (tid == 0) {
            const double elapsed = 1e-9 * (double)(now_ns() - t_start);
            bc_restart = 0;
            bc_stop = 0;
            if (is_r0 && !is_check) {
                R0 = Rt;
                Rprev = Rt;
                if (nrec < A.rec_cap) {
                    hpr_check_record rec{};
                    rec.k = k; rec.r = r; rec.t = 0; rec.kind = 2; rec.cause = 0;
                    rec.sigma = sigma; rec.Rt = R0; rec.R0 = R0; rec.sigma_next = sigma;
                    rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = sigma;
                    A.recs[nrec] = rec;
                }
                ++nrec;
            } else {
                if (is_r0) {
                    R0 = Rt;
                    Rprev = Rt;
                }
                // termination test of Section 4.1 in the original space
                const double bb = A.beta_b * A.beta_c;
                errp = sqrt(S_RP) / (1.0 + A.norm_b);
                errd = sqrt(S_RD) / (1.0 + A.norm_c);
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
                } else if (kkt <= A.tol) {
                    status = 0;
                    cause = -1;
                    bc_stop = 1;
                } else if (k + 1 < A.max_iter && A.restart && !is_r0) {
                    // restart criteria eq. (restart_1)-(restart_3)
                    if (Rt <= A.alpha1 * R0) cause = 1;
                    else if (Rt <= A.alpha2 * R0 && Rt > Rprev) cause = 2;
                    else if ((double)(t_all + 1) >= A.alpha3 * (double)(k + 1)) cause = 3;
                    Rprev = Rt;
                    bc_restart = cause != 0;
                }
                if (bc_restart) {
                    // Algorithm 3 with eq. (sigma_T1!=0)
                    Dx = sqrt(S_XX0);
                    Dy = sqrt(lambda) * sqrt(S_YY0);
                    const double ratio = errd / errp;
                    if (A.sigma_update && Dx > 1e-16 && Dx < 1e12 && Dy > 1e-16 && Dy < 1e12 && errp > 0.0 &&
                        ratio > 1e-8 && ratio < 1e8)
                        sigma_next = Dx / Dy;
                    else
                        sigma_next = A.sigma_update ? 1.0 : sigma;
                }
                if (nrec < A.rec_cap) {
                    hpr_check_record rec{};
                    rec.k = k; rec.r = r; rec.t = t_all; rec.kind = 1 + (is_r0 ? 2 : 0); rec.cause = cause;
                    rec.sigma = sigma; rec.err_p = errp; rec.err_d = errd; rec.err_gap = gap; rec.kkt = kkt;
                    rec.pobj = pobj; rec.dobj = dobj; rec.Rt = Rt; rec.R0 = R0; rec.sigma_next = sigma_next;
                    rec.Dx = Dx; rec.Dy = Dy; rec.elapsed_s = elapsed; rec.action = -1; rec.sigma_rule = sigma_next;
                    A.recs[nrec] = rec;
                }
                ++nrec;
                if (bc_restart) {
                    bc_sigma = sigma_next;
                    ++r;
                }
            }
        }
        if (tid == 0) next_scalars(bc_restart ? 0 : t_all + 1);
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
    // the last w_bar into the multi-CTA path's renumbered arrays (for its back-map)
    for (int j = tid; j < n; j += NT) {
        const int o = A.perm_c[j];
        A.xbar_out[j] = xb[o];
        A.zbar_out[j] = zb[o];
    }
    for (int i = tid; i < m; i += NT) A.ybar_out[i] = yb[A.perm_r[i]];
    if (tid == 0) {
        double *o = A.out;
        o[SO_ITERS] = (double)k; o[SO_RESTARTS] = (double)r; o[SO_STATUS] = (double)status;
        o[SO_LAMBDA] = lambda; o[SO_POWER_ITERS] = (double)piters; o[SO_SIGMA] = bc_sigma;
        o[SO_POBJ] = pobj; o[SO_DOBJ] = dobj; o[SO_ERRP] = errp; o[SO_ERRD] = errd; o[SO_GAP] = gap;
        o[SO_KKT] = kkt; o[SO_T1E4] = t1e4; o[SO_I1E4] = (double)i1e4; o[SO_NREC] = (double)nrec;
        o[SO_POWER_S] = 1e-9 * (double)(t_power - t_start);
        o[SO_TOTAL_S] = 1e-9 * (double)(now_ns() - t_start);
    }
}

}  // namespace hprsmall
